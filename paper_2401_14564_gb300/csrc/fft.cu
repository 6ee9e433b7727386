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
// a CTA transforms a tile of neighbouring lines (rows along x, columns along y
// and z, so every global access is a row of consecutive complex values); the
// first stage reads global memory, the last writes it, the ones between
// exchange through shared memory.
#include <cuda_runtime.h>

#include "pp_internal.cuh"

namespace pp {
namespace {

constexpr int kFftThreads = 256;  // 4 CTAs per SM at 64 registers, tiles of up to 36 KB
constexpr int kFftBlocksPerSm = 4;
constexpr int kUnits = 2;          // stage units per thread per trip
constexpr int kLines = 16;         // lines per tile along x (at most)
constexpr int kStridedLines = 64;  // columns per tile along y and z (at most)

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

// A pass transforms tiles of nl = 2^log2nl lines of n = 2^LOG2N elements.  kContig: lines along x
// (element p of line l at base + l lstride + p); else columns along y or z (at base + l +
// p pstride).  In shared memory, columns are interleaved (element p of line l at p nl + l:
// consecutive threads take consecutive lines, so a warp touches consecutive banks).  Rows lie
// one after the other, element e = l n + p, in a layout chosen by the stage that writes them so
// that both its writes and the next stage's reads (runs of 16 consecutive elements) spread over
// the 32 banks (a complex value spans two): after the first radix-8 stage (stride-8 writes) the
// low 3 bits of e are XORed with bits 4-6; after the second (runs of 8 at stride 64) every 64
// elements are followed by 8 pad slots; later stages write runs of 16 or more and keep e.  n is
// a template parameter: every stage's index arithmetic folds to shifts and masks of constants.
struct Pass {
    int log2nl, nbi, ntiles;
    long long outer_pitch, stride;  // stride: lstride for rows, pstride for columns
    long long limit;                // complex values in the array (index bound)
    float sign;
};

template <int LOG2N, bool kContig>
struct TileAt {
    long long base, stride, limit;
    int log2nl;
    __device__ __forceinline__ long long at(int l, int p) const {
        return checked(kContig ? base + l * stride + p : base + l + p * stride, limit, kChkFft);
    }
    // slot of element p of line l in the layout written by the stage after radices L = 2^LOG2W
    template <int LOG2W>
    __device__ __forceinline__ int slot(int l, int p) const {
        if (!kContig) return (p << log2nl) + l;
        const int e = (l << LOG2N) + p;
        if constexpr (LOG2W == 0) return e ^ ((e >> 4) & 7);
        else if constexpr (LOG2W == 3) return e + 8 * (e >> 6);
        else return e;
    }
};

// Slots of the largest layout (8 pad slots per 64 elements along rows).
template <int LOG2N, bool kContig>
__host__ __device__ __forceinline__ int tile_slots(int nl) {
    return kContig ? (nl << LOG2N) + (nl << LOG2N) / 8 : nl << LOG2N;
}

// Twiddles of the stage after radices L = 2^LOG2L (all radix 8 before it), radix R = 2^LR:
// w_{LR}^{m j} for m = 1..R-1, j = 0..L-1 at tw[(L - 1) + (m - 1) L + j], so that threads with
// consecutive j read consecutive slots; the stages' tables together fill tw[0 .. n-2].
template <int LOG2L, int LR>
__device__ __forceinline__ void stage_twiddles(float2* tw, float sign) {
    constexpr int L = 1 << LOG2L, R = 1 << LR;
    for (int e = threadIdx.x; e < (R - 1) * L; e += kFftThreads) {
        const int m = (e >> LOG2L) + 1, j = e & (L - 1);
        float sn, cs;
        sincospif((float)(m * j) * (2.f / (float)(L * R)), &sn, &cs);
        tw[(L - 1) + e] = make_float2(cs, sign * sn);
    }
}

// One Stockham stage of radix R = 2^LR after stages whose radices multiply to L = 2^LOG2L: unit
// (line l, t), t < n/R, j = t mod L, k = t / L, reads a_m = x[t + m n/R], twiddles a_m by
// w_{LR}^{m j}, transforms, writes y[k L R + j + m L].  kFirst reads global memory, kLast
// writes it; the others read and write the tile in place (every read of a stage precedes its
// writes: a stage that writes the tile runs in one trip, see lines_per_block).
template <int LOG2N, bool kContig, int LR, int LOG2L, bool kFirst, bool kLast>
__device__ __forceinline__ void stage(float2* data, const TileAt<LOG2N, kContig>& T, float2* x, const float2* tw,
                                      float sign) {
    constexpr int R = 1 << LR, LOG2NR = LOG2N - LR, NR = 1 << LOG2NR;
    const int units = 1 << (T.log2nl + LOG2NR);
    const int nl_mask = (1 << T.log2nl) - 1;
    constexpr int U = kUnits;
    for (int u0 = 0; u0 < units; u0 += kFftThreads * U) {
        float2 a[U][R];
        int ul[U], ut[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int u = u0 + q * kFftThreads + threadIdx.x;
            // consecutive threads: consecutive t along rows, consecutive lines across columns
            ul[q] = kContig ? u >> LOG2NR : u & nl_mask;
            ut[q] = kContig ? u & (NR - 1) : u >> T.log2nl;
            if (u < units) {
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const int p = ut[q] + m * NR;
                    if constexpr (kFirst) a[q][m] = data[T.at(ul[q], p)];
                    else a[q][m] = x[T.template slot<LOG2L - 3>(ul[q], p)];
                }
            }
        }
        if (!kFirst) __syncthreads();
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int u = u0 + q * kFftThreads + threadIdx.x;
            if (u >= units) continue;
            const int t = ut[q], j = t & ((1 << LOG2L) - 1), k = t >> LOG2L;
#pragma unroll
            for (int m = 1; m < R; ++m) a[q][m] = cmul(tw[((1 << LOG2L) - 1) + ((m - 1) << LOG2L) + j], a[q][m]);
            dft<R>(a[q], sign);
#pragma unroll
            for (int m = 0; m < R; ++m) {
                const int p = (k << (LOG2L + LR)) + j + (m << LOG2L);
                if constexpr (kLast) data[T.at(ul[q], p)] = a[q][m];
                else x[T.template slot<LOG2L>(ul[q], p)] = a[q][m];
            }
        }
        if (!kLast) __syncthreads();
    }
}

// All stages of one tile: radix-8 stages first (the first reading global memory), the radix-2
// or radix-4 remainder last.
template <int LOG2N, bool kContig>
__device__ __forceinline__ void fft_tile(float2* data, const TileAt<LOG2N, kContig>& T, float2* x, const float2* tw,
                                         float sign) {
    constexpr int N8 = LOG2N / 3, REST = LOG2N - 3 * N8;
    if constexpr (N8 >= 1) stage<LOG2N, kContig, 3, 0, true, N8 == 1 && REST == 0>(data, T, x, tw, sign);
    if constexpr (N8 >= 2) stage<LOG2N, kContig, 3, 3, false, N8 == 2 && REST == 0>(data, T, x, tw, sign);
    if constexpr (N8 >= 3) stage<LOG2N, kContig, 3, 6, false, N8 == 3 && REST == 0>(data, T, x, tw, sign);
    if constexpr (REST == 1) stage<LOG2N, kContig, 1, 3 * N8, N8 == 0, true>(data, T, x, tw, sign);
    if constexpr (REST == 2) stage<LOG2N, kContig, 2, 3 * N8, N8 == 0, true>(data, T, x, tw, sign);
}

// One 1D pass: CTA b takes tile b, i.e. outer index b / nbi and lines (b % nbi) nl onwards, at
// (b / nbi) outer_pitch + line lstride + p pstride (see fft3 for the three axes of the padded
// layout).  sign = -1 forward, +1 inverse (unnormalised).
template <int LOG2N, bool kContig>
__global__ void __launch_bounds__(kFftThreads, kFftBlocksPerSm) fft_pass_kernel(float2* data, const Pass P) {
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int N = 1 << LOG2N;
    float2* tw = reinterpret_cast<float2*>(smraw);  // the stages' twiddle tables, N - 1 values
    float2* x = tw + N;
    constexpr int N8 = LOG2N / 3, REST = LOG2N - 3 * N8;
    if constexpr (N8 >= 1) stage_twiddles<0, 3>(tw, P.sign);
    if constexpr (N8 >= 2) stage_twiddles<3, 3>(tw, P.sign);
    if constexpr (N8 >= 3) stage_twiddles<6, 3>(tw, P.sign);
    if constexpr (REST > 0) stage_twiddles<3 * N8, REST>(tw, P.sign);
    TileAt<LOG2N, kContig> T;
    const int b = blockIdx.x;
    T.base = (long long)(b / P.nbi) * P.outer_pitch + ((long long)(b % P.nbi) << P.log2nl) * (kContig ? P.stride : 1);
    T.stride = P.stride;
    T.limit = P.limit;
    T.log2nl = P.log2nl;
    __syncthreads();
    fft_tile<LOG2N, kContig>(data, T, x, tw, P.sign);
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
// Rows of nx >= 4 go four nodes per thread: two 16-byte loads, two 16-byte stores (row starts
// are 16-byte aligned on both sides: nx, nx + 16 and the plane pitch are multiples of 4).
__global__ void pack_kernel(const float* __restrict__ f, const float* __restrict__ g, float2* z, const Pad P, float p) {
    const int rows = P.ny * P.nz;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int j = r % P.ny, k = r / P.ny;
        const long long src = (long long)r * P.nx, dst = P.at(0, j, k);
        // the row's last complex value and last input float lie inside their arrays
        checked(dst + P.nx - 1, (long long)P.nz * P.pz, kChkFft);
        checked(src + P.nx - 1, (long long)P.nx * P.ny * P.nz, kChkFft);
        if ((P.nx & 3) == 0) {
            const float4* f4 = reinterpret_cast<const float4*>(f + src);
            const float4* g4 = reinterpret_cast<const float4*>(g + src);
            float4* z4 = reinterpret_cast<float4*>(z + dst);
            for (int i = threadIdx.x; i < (P.nx >> 2); i += blockDim.x) {
                const float4 a = __ldg(f4 + i), b = __ldg(g4 + i);
                z4[2 * i] = make_float4(powered(a.x, p), powered(b.x, p), powered(a.y, p), powered(b.y, p));
                z4[2 * i + 1] = make_float4(powered(a.z, p), powered(b.z, p), powered(a.w, p), powered(b.w, p));
            }
        } else {
            for (int i = threadIdx.x; i < P.nx; i += blockDim.x)
                z[dst + i] = make_float2(powered(__ldg(f + src + i), p), powered(__ldg(g + src + i), p));
        }
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
        const long long row = checked(P.at(0, j, k), (long long)P.nz * P.pz - P.nx + 1, kChkFft);
        const long long mrow = checked(P.at(0, mj, mk), (long long)P.nz * P.pz - P.nx + 1, kChkFft);
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
        const long long src = checked(P.at(0, r % P.ny, r / P.ny), (long long)P.nz * P.pz - P.nx + 1, kChkFft);
        const long long dst = checked((long long)r * P.nx, (long long)P.nx * P.ny * P.nz - P.nx + 1, kChkFft);
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

template <int LOG2N, bool kContig>
cudaError_t launch_pass(float2* data, const Pass& P, cudaStream_t s) {
    const size_t smem = ((size_t)(1 << LOG2N) + (size_t)tile_slots<LOG2N, kContig>(1 << P.log2nl)) * sizeof(float2);
    auto k = fft_pass_kernel<LOG2N, kContig>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<P.ntiles, kFftThreads, smem, s>>>(data, P);
    return cudaGetLastError();
}

template <bool kContig>
cudaError_t launch_pass_n(float2* data, int log2n, const Pass& P, cudaStream_t s) {
    switch (log2n) {
        case 1: return launch_pass<1, kContig>(data, P, s);
        case 2: return launch_pass<2, kContig>(data, P, s);
        case 3: return launch_pass<3, kContig>(data, P, s);
        case 4: return launch_pass<4, kContig>(data, P, s);
        case 5: return launch_pass<5, kContig>(data, P, s);
        case 6: return launch_pass<6, kContig>(data, P, s);
        case 7: return launch_pass<7, kContig>(data, P, s);
        case 8: return launch_pass<8, kContig>(data, P, s);
        case 9: return launch_pass<9, kContig>(data, P, s);
        case 10: return launch_pass<10, kContig>(data, P, s);
        default: return cudaErrorInvalidValue;
    }
}

// Tiles of nl lines of n; nbi tiles per outer index; rows along x (lines lstride apart) or columns
// (elements pstride apart).
cudaError_t fft_axis(float2* data, long long limit, bool rows, int n, int nl, int nbi, int nouter,
                     long long outer_pitch, long long stride, float sign, cudaStream_t s) {
    if (n < 2) return cudaSuccess;
    Pass P;
    P.log2nl = ilog2i(nl);
    P.nbi = nbi;
    P.ntiles = nbi * nouter;
    P.outer_pitch = outer_pitch;
    P.stride = stride;
    P.limit = limit;
    P.sign = sign;
    return rows ? launch_pass_n<true>(data, ilog2i(n), P, s) : launch_pass_n<false>(data, ilog2i(n), P, s);
}

// Lines per tile for lines of n among `avail` neighbours: up to `want`, fewer when the axis
// has fewer, and at most 8 U kFftThreads / n (U units per thread) so that a radix-8 stage that
// writes shared memory (in place) has at most U kFftThreads units: all of its reads then happen
// before its writes.
int lines_per_block(int n, int avail, int want, int units) {
    const int cap = 8 * units * kFftThreads / n;
    const int L = avail < want ? avail : want;
    return L < cap ? L : cap;
}

cudaError_t fft3(float2* data, const Pad& P, float sign, cudaStream_t s) {
    cudaError_t e;
    int nl = lines_per_block(P.nx, P.ny, kLines, kUnits);  // x: lines are rows j of a plane k
    const long long lim = (long long)P.nz * P.pz;
    if ((e = fft_axis(data, lim, true, P.nx, nl, P.ny / nl, P.nz, P.pz, P.px, sign, s)) != cudaSuccess) return e;
    nl = lines_per_block(P.ny, P.nx, kStridedLines, kUnits);  // y: lines are columns i of a plane k
    if ((e = fft_axis(data, lim, false, P.ny, nl, P.nx / nl, P.nz, P.pz, P.px, sign, s)) != cudaSuccess) return e;
    nl = lines_per_block(P.nz, P.nx, kStridedLines, kUnits);  // z: lines are columns i of a row j
    return fft_axis(data, lim, false, P.nz, nl, P.nx / nl, P.ny, P.px, P.pz, sign, s);
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

PP_CHECK_READER(check_flags_fft)

}  // namespace pp
