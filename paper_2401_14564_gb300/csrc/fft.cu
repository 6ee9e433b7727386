// Cross-correlation force fields (Eqs. El_conv and Pauli_FDBM; Sec. 5.1.2:
// the convolution theorem turns the correlation into a product in Fourier
// space).  For a sample field f and a tip density g on the same periodic grid,
//   E[n] = scale * dV * sum_h g[h]^p f[n + h]^p,   F = -grad E,
// with the gradient taken spectrally (i k, Nyquist terms dropped so that the
// force stays real).  Steps, all in this file:
//   pack      z = f^p + i g^p (two real transforms in one complex one);
//   fft3      forward 3D FFT of z: 1D passes along x, y and z;
//   spectral  F^ = (Z_k + Z*_-k)/2, G^ = (Z_k - Z*_-k)/(2i), P = G^* F^ scale dV / N,
//             B1 = P + i(-i kx P), B2 = (-i ky P) + i(-i kz P);
//   fft3      inverse 3D FFTs of B1 and B2 -> (E, Fx) and (Fy, Fz) as (re, im);
//   output    ff[n] = (Fx, Fy, Fz, E), written or added.
// The 1D passes are Stockham auto-sort FFTs with radix-8 stages (and one
// radix-2 or radix-4 stage) in registers, for power-of-two lengths up to 1024:
// the first stage reads global memory, the last writes it, the ones between
// exchange through shared memory; a block transforms 16 lines, and along y
// and z those are 16 neighbouring columns, so every global access is a row of
// consecutive complex values.
#include <cuda_runtime.h>

#include "pp_internal.cuh"

namespace pp {
namespace {

constexpr int kFftThreads = 512;  // 2 blocks per SM at 64 registers: 32 warps to keep loads in flight
constexpr int kUnits = 2;         // stage units per thread per trip
constexpr int kLines = 16;         // lines per block along x
constexpr int kStridedLines = 64;  // columns per block along y and z (at most)

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// In-register DFT of R points (R = 2, 4, 8), natural order, w = exp(sign 2 pi i / R).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul_i(float2 a, float sign) { return make_float2(-sign * a.y, sign * a.x); }

template <int R>
__device__ __forceinline__ void dft(float2 (&x)[R], float sign);

template <>
__device__ __forceinline__ void dft<2>(float2 (&x)[2], float) {
    const float2 a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void dft<4>(float2 (&x)[4], float sign) {
    const float2 t0 = cadd(x[0], x[2]), t1 = csub(x[0], x[2]);
    const float2 t2 = cadd(x[1], x[3]), t3 = mul_i(csub(x[1], x[3]), sign);
    x[0] = cadd(t0, t2);
    x[2] = csub(t0, t2);
    x[1] = cadd(t1, t3);
    x[3] = csub(t1, t3);
}

template <>
__device__ __forceinline__ void dft<8>(float2 (&x)[8], float sign) {
    float2 e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
    dft<4>(e, sign);
    dft<4>(o, sign);
    const float h = 0.70710678118654752f;  // w8 = h (1 + sign i)
    const float2 o1 = make_float2(h * (o[1].x - sign * o[1].y), h * (o[1].y + sign * o[1].x));
    const float2 o2 = mul_i(o[2], sign);
    const float2 o3 = make_float2(h * (-o[3].x - sign * o[3].y), h * (-o[3].y + sign * o[3].x));  // w8^3 = h(-1 + sign i)
    x[0] = cadd(e[0], o[0]);
    x[4] = csub(e[0], o[0]);
    x[1] = cadd(e[1], o1);
    x[5] = csub(e[1], o1);
    x[2] = cadd(e[2], o2);
    x[6] = csub(e[2], o2);
    x[3] = cadd(e[3], o3);
    x[7] = csub(e[3], o3);
}

// Address of element p of line l within a block: base + l * lstride + p * pstride.
struct Lines {
    long long base;
    long long lstride, pstride;
    bool contiguous;  // pstride == 1: consecutive threads take consecutive elements of a line
    __device__ __forceinline__ long long at(int l, int p) const { return base + l * lstride + p * pstride; }
};

// Shared-memory slot of element p of line l: lines one after the other when
// consecutive threads walk along a line, interleaved when they walk across
// lines (strided passes), so that a warp's accesses hit consecutive banks.
__device__ __forceinline__ int sidx(const Lines& ln, int l, int p, int n, int nl) {
    return ln.contiguous ? l * n + p : p * nl + l;
}

// One Stockham stage of radix R with L = product of the earlier radices: unit
// (line l, t), t < n/R, j = t mod L, k = t / L, reads a_m = x[t + m n/R],
// twiddles a_m by w_{LR}^{m j}, transforms, writes y[k L R + j + m L].  The
// first stage reads global memory, the last writes it, the others work in
// shared memory (in place: every read of a stage precedes its writes).
template <int R>
__device__ __forceinline__ void stockham_stage(float2* data, const Lines& ln, float2* x, const float2* tw, int n,
                                               int nlines, int L, bool first, bool last, float sign) {
    const int nr = n / R, units = nlines * nr;
    const int tws = n / (L * R);
    // middle stages (neither first nor last) have units <= kUnits * kFftThreads: one trip
    for (int u0 = 0; u0 < units; u0 += kFftThreads * kUnits) {
        float2 a[kUnits][R];
        int ul[kUnits], ut[kUnits];
#pragma unroll
        for (int q = 0; q < kUnits; ++q) {
            const int u = u0 + q * kFftThreads + threadIdx.x;
            // consecutive threads: consecutive t for contiguous lines, consecutive lines otherwise
            ul[q] = ln.contiguous ? u / nr : u % nlines;
            ut[q] = ln.contiguous ? u - ul[q] * nr : u / nlines;
            if (u < units) {
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const int p = ut[q] + m * nr;
                    a[q][m] = first ? data[ln.at(ul[q], p)] : x[sidx(ln, ul[q], p, n, nlines)];
                }
            }
        }
        if (!first) __syncthreads();
#pragma unroll
        for (int q = 0; q < kUnits; ++q) {
            const int u = u0 + q * kFftThreads + threadIdx.x;
            if (u >= units) continue;
            const int t = ut[q], j = t % L, k = t / L;
#pragma unroll
            for (int m = 1; m < R; ++m) a[q][m] = cmul(tw[m * j * tws], a[q][m]);
            dft<R>(a[q], sign);
#pragma unroll
            for (int m = 0; m < R; ++m) {
                const int p = k * L * R + j + m * L;
                if (last) data[ln.at(ul[q], p)] = a[q][m];
                else x[sidx(ln, ul[q], p, n, nlines)] = a[q][m];
            }
        }
        if (!last) __syncthreads();
    }
}

// One 1D pass: block b transforms nl lines of n elements, element p of line
// l at (b / nbi) * outer_pitch + (b % nbi) * nl * lstride + l * lstride +
// p * pstride (see fft3 for the three axes of the padded layout).  sign = -1
// forward, +1 inverse (unnormalised).  Radix-8 stages, then one radix-4 or
// radix-2 stage for the rest of log2 n.
__global__ void __launch_bounds__(kFftThreads, 2) fft_pass_kernel(float2* data, int n, int log2n, int nl, int nbi,
                                                                  long long outer_pitch, long long lstride,
                                                                  long long pstride, float sign) {
    extern __shared__ float2 sm[];
    float2* tw = sm;      // n twiddles exp(sign 2 pi i q / n)
    float2* x = sm + n;   // nl lines of n
    for (int q = threadIdx.x; q < n; q += kFftThreads) {
        float s, c;
        sincospif(2.f * (float)q / (float)n, &s, &c);
        tw[q] = make_float2(c, sign * s);
    }
    Lines ln;
    ln.base = (long long)(blockIdx.x / nbi) * outer_pitch + (long long)(blockIdx.x % nbi) * nl * lstride;
    ln.lstride = lstride;
    ln.pstride = pstride;
    ln.contiguous = pstride == 1;
    __syncthreads();
    // radix-8 stages first (the first stage, read from global memory, then has 8 loads per
    // unit in flight), the radix-2 or radix-4 remainder last
    const int n8 = log2n / 3, rest = log2n - 3 * n8;
    const int nstages = n8 + (rest ? 1 : 0);
    int L = 1;
    for (int s = 0; s < n8; ++s) {
        stockham_stage<8>(data, ln, x, tw, n, nl, L, s == 0, s == nstages - 1, sign);
        L <<= 3;
    }
    if (rest == 1) stockham_stage<2>(data, ln, x, tw, n, nl, L, n8 == 0, true, sign);
    else if (rest == 2) stockham_stage<4>(data, ln, x, tw, n, nl, L, n8 == 0, true, sign);
}

__device__ __forceinline__ float powered(float v, float p) {
    if (p == 1.f) return v;
    return v > 0.f ? powf(v, p) : 0.f;
}

// Padded complex layout of the scratch arrays: node (i, j, k) at
// k * pz + j * px + i with px = nx + 16 and pz = px * ny + 16, so that the
// strides of the y and z passes are not powers of two (a power-of-two stride
// sends every row of a pass to the same memory channels) while every row stays
// 128-byte aligned.
struct Pad {
    int nx, ny, nz;
    long long px, pz;
    __device__ __forceinline__ long long at(int i, int j, int k) const { return (long long)k * pz + (long long)j * px + i; }
};

Pad make_pad(int nx, int ny, int nz) {
    Pad P;
    P.nx = nx; P.ny = ny; P.nz = nz;
    P.px = nx + 16;
    P.pz = P.px * ny + 16;
    return P;
}

// Elementwise kernels walk rows (j, k) of the grid: blocks take rows, threads the
// x index, so no per-element division is needed.
__global__ void pack_kernel(const float* __restrict__ f, const float* __restrict__ g, float2* z, const Pad P, float p) {
    const int rows = P.ny * P.nz;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int j = r % P.ny, k = r / P.ny;
        const long long src = (long long)r * P.nx, dst = P.at(0, j, k);
        for (int i = threadIdx.x; i < P.nx; i += blockDim.x)
            z[dst + i] = make_float2(powered(__ldg(f + src + i), p), powered(__ldg(g + src + i), p));
    }
}

struct SpecArgs {
    const float2* z;
    float2 *b1, *b2;
    Pad P;
    float kx0, ky0, kz0;  // 2 pi / (n d) per axis
    float norm;           // scale * dV / N
};

// Wavenumber of index m along an axis of length n (Nyquist -> 0 for the derivative).
__device__ __forceinline__ float wavenumber(int m, int n, float k0) {
    if (2 * m == n) return 0.f;
    return (2 * m < n ? (float)m : (float)(m - n)) * k0;
}

__global__ void spectral_kernel(const SpecArgs A) {
    const Pad& P = A.P;
    const int rows = P.ny * P.nz;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int j = r % P.ny, k = r / P.ny;
        const int mj = j == 0 ? 0 : P.ny - j, mk = k == 0 ? 0 : P.nz - k;
        const float ky = wavenumber(j, P.ny, A.ky0), kz = wavenumber(k, P.nz, A.kz0);
        const long long row = P.at(0, j, k), mrow = P.at(0, mj, mk);
        for (int i = threadIdx.x; i < P.nx; i += blockDim.x) {
            const int mi = i == 0 ? 0 : P.nx - i;
            const float2 zk = A.z[row + i];
            const float2 zm = A.z[mrow + mi];
            // F^ = (Z_k + conj Z_-k)/2, G^ = (Z_k - conj Z_-k)/(2i)
            const float2 F = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            const float2 G = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
            // P = conj(G) F * norm
            const float2 Pk = make_float2(A.norm * fmaf(G.x, F.x, G.y * F.y), A.norm * fmaf(G.x, F.y, -G.y * F.x));
            const float kx = wavenumber(i, P.nx, A.kx0);
            // -i k P = (k P.y, -k P.x); B1 = P + i(-i kx P), B2 = (-i ky P) + i(-i kz P); i (a + ib) = (-b, a)
            const float2 dx = make_float2(kx * Pk.y, -kx * Pk.x);
            const float2 dy = make_float2(ky * Pk.y, -ky * Pk.x);
            const float2 dz = make_float2(kz * Pk.y, -kz * Pk.x);
            A.b1[row + i] = make_float2(Pk.x - dx.y, Pk.y + dx.x);
            A.b2[row + i] = make_float2(dy.x - dz.y, dy.y + dz.x);
        }
    }
}

__global__ void output_kernel(const float2* __restrict__ b1, const float2* __restrict__ b2, float4* ff, const Pad P,
                              int accumulate) {
    const int rows = P.ny * P.nz;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const long long src = P.at(0, r % P.ny, r / P.ny), dst = (long long)r * P.nx;
        for (int i = threadIdx.x; i < P.nx; i += blockDim.x) {
            const float2 a = b1[src + i], b = b2[src + i];  // (E, Fx), (Fy, Fz)
            float4 v = make_float4(a.y, b.x, b.y, a.x);     // the spectra already hold -i k P: forces
            if (accumulate) {
                const float4 w = ff[dst + i];
                v = make_float4(w.x + v.x, w.y + v.y, w.z + v.z, w.w + v.w);
            }
            ff[dst + i] = v;
        }
    }
}

int ilog2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// nl lines of n per block; lines of the block are lstride apart, blocks nbi per outer index.
cudaError_t fft_axis(float2* data, int n, int nl, int nbi, int nouter, long long outer_pitch, long long lstride,
                     long long pstride, float sign, cudaStream_t s) {
    if (n < 2) return cudaSuccess;
    const size_t smem = (size_t)(n + nl * n) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fft_pass_kernel<<<nouter * nbi, kFftThreads, smem, s>>>(data, n, ilog2i(n), nl, nbi, outer_pitch, lstride, pstride,
                                                           sign);
    return cudaGetLastError();
}

// Lines per block for lines of n among `avail` neighbours: up to `want`, fewer when the axis
// has fewer, and at most 8 kUnits kFftThreads / n so that a middle (shared-memory, in-place)
// radix-8 stage has at most kUnits * kFftThreads units: all of its reads then happen before
// its writes.  Strided passes take up to 64 columns (512-byte rows), so that each of the n
// widely spaced rows a block visits is read in one long burst.
int lines_per_block(int n, int avail, int want) {
    int L = avail < want ? avail : want;
    return L < 8 * kUnits * kFftThreads / n ? L : 8 * kUnits * kFftThreads / n;
}

cudaError_t fft3(float2* data, const Pad& P, float sign, cudaStream_t s) {
    cudaError_t e;
    int nl = lines_per_block(P.nx, P.ny, kLines);  // x: lines are rows j of a plane k
    if ((e = fft_axis(data, P.nx, nl, P.ny / nl, P.nz, P.pz, P.px, 1, sign, s)) != cudaSuccess) return e;
    nl = lines_per_block(P.ny, P.nx, kStridedLines);  // y: lines are columns i of a plane k
    if ((e = fft_axis(data, P.ny, nl, P.nx / nl, P.nz, P.pz, 1, P.px, sign, s)) != cudaSuccess) return e;
    nl = lines_per_block(P.nz, P.nx, kStridedLines);  // z: lines are columns i of a row j
    return fft_axis(data, P.nz, nl, P.nx / nl, P.ny, P.px, 1, P.pz, sign, s);
}

}  // namespace

size_t fft_workspace_bytes(int nx, int ny, int nz) {
    const Pad P = make_pad(nx, ny, nz);
    return (size_t)3 * (size_t)(P.nz * P.pz) * sizeof(float2);
}

cudaError_t launch_fft_correlate(const FftLaunch& L, cudaStream_t s) {
    const Pad P = make_pad(L.nx, L.ny, L.nz);
    const long long N = (long long)L.nx * L.ny * L.nz, NP = (long long)P.nz * P.pz;
    float2* z = reinterpret_cast<float2*>(L.ws);
    float2* b1 = z + NP;
    float2* b2 = b1 + NP;
    const int threads = 256;
    const int rows = L.ny * L.nz;
    const int blocks = rows < 152 * 32 ? rows : 152 * 32;
    pack_kernel<<<blocks, threads, 0, s>>>(L.f, L.g, z, P, L.power);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = fft3(z, P, -1.f, s)) != cudaSuccess) return e;
    SpecArgs A;
    A.z = z;
    A.b1 = b1;
    A.b2 = b2;
    A.P = P;
    A.kx0 = (float)(2.0 * kPi / (L.nx * (double)L.dx));
    A.ky0 = (float)(2.0 * kPi / (L.ny * (double)L.dy));
    A.kz0 = (float)(2.0 * kPi / (L.nz * (double)L.dz));
    A.norm = (float)((double)L.scale * (double)L.dx * L.dy * L.dz / (double)N);
    spectral_kernel<<<blocks, threads, 0, s>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = fft3(b1, P, 1.f, s)) != cudaSuccess) return e;
    if ((e = fft3(b2, P, 1.f, s)) != cudaSuccess) return e;
    output_kernel<<<blocks, threads, 0, s>>>(b1, b2, L.ff, P, L.accumulate);
    return cudaGetLastError();
}

}  // namespace pp
