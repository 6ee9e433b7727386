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
// The 1D passes are radix-2 decimation in time in shared memory, with a
// twiddle table per block, for power-of-two lengths up to 1024: a block
// transforms 16 lines; along y and z the lines are 16 neighbouring columns so
// that every global access is a row of consecutive complex values.
#include <cuda_runtime.h>

#include "pp_internal.cuh"

namespace pp {
namespace {

constexpr int kFftThreads = 256;
constexpr int kLines = 16;  // lines per block

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ int bitrev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

// One 1D pass over a [outer][n][inner] view of the array: line (o, c) holds
// elements o*n*inner + p*inner + c, p = 0..n-1.  A block takes kLines
// consecutive columns c (or, for inner = 1, kLines consecutive lines o).
// sign = -1 forward, +1 inverse (unnormalised).
__global__ void __launch_bounds__(kFftThreads) fft_pass_kernel(float2* data, int n, int log2n, int inner,
                                                               int lines_per_block, int nblocks_inner, float sign) {
    extern __shared__ float2 sm[];
    float2* tw = sm;                 // n/2 twiddles exp(sign 2 pi i j / n)
    float2* x = sm + (n >> 1);       // lines_per_block lines of n, bit-reversed order
    const int L = lines_per_block;
    for (int j = threadIdx.x; j < (n >> 1); j += kFftThreads) {
        float s, c;
        sincospif(2.f * (float)j / (float)n, &s, &c);
        tw[j] = make_float2(c, sign * s);
    }
    // this block's lines
    const long long o = inner == 1 ? (long long)blockIdx.x * L : blockIdx.x / nblocks_inner;
    const int c0 = inner == 1 ? 0 : (blockIdx.x % nblocks_inner) * L;
    const long long base = inner == 1 ? o * n : o * (long long)n * inner + c0;
    // load: element p of line l -> x[l*n + bitrev(p)]; consecutive threads read consecutive addresses
    for (int t = threadIdx.x; t < L * n; t += kFftThreads) {
        int l, p;
        long long addr;
        if (inner == 1) {
            l = t / n;
            p = t - l * n;
            addr = base + (long long)l * n + p;
        } else {
            p = t / L;
            l = t - p * L;
            addr = base + (long long)p * inner + l;
        }
        x[l * n + bitrev(p, log2n)] = data[addr];
    }
    __syncthreads();
    const int half_total = L * (n >> 1);
    for (int s = 0; s < log2n; ++s) {
        const int half = 1 << s, len = half << 1;
        const int tstride = n >> (s + 1);  // twiddle index step at this length
        for (int b = threadIdx.x; b < half_total; b += kFftThreads) {
            const int l = b / (n >> 1), r = b - l * (n >> 1);
            const int grp = r >> s, pos = r & (half - 1);
            float2* xl = x + l * n;
            const int i0 = grp * len + pos, i1 = i0 + half;
            const float2 u = xl[i0];
            const float2 v = cmul(tw[pos * tstride], xl[i1]);
            xl[i0] = make_float2(u.x + v.x, u.y + v.y);
            xl[i1] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < L * n; t += kFftThreads) {
        int l, p;
        long long addr;
        if (inner == 1) {
            l = t / n;
            p = t - l * n;
            addr = base + (long long)l * n + p;
        } else {
            p = t / L;
            l = t - p * L;
            addr = base + (long long)p * inner + l;
        }
        data[addr] = x[l * n + p];
    }
}

__device__ __forceinline__ float powered(float v, float p) {
    if (p == 1.f) return v;
    return v > 0.f ? powf(v, p) : 0.f;
}

__global__ void pack_kernel(const float* __restrict__ f, const float* __restrict__ g, float2* z, long long N, float p) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x)
        z[q] = make_float2(powered(__ldg(f + q), p), powered(__ldg(g + q), p));
}

struct SpecArgs {
    const float2* z;
    float2 *b1, *b2;
    int nx, ny, nz;
    float kx0, ky0, kz0;  // 2 pi / (n d) per axis
    float norm;           // scale * dV / N
};

// Wavenumber of index m along an axis of length n (Nyquist -> 0 for the derivative).
__device__ __forceinline__ float wavenumber(int m, int n, float k0) {
    if (2 * m == n) return 0.f;
    return (2 * m < n ? (float)m : (float)(m - n)) * k0;
}

__global__ void spectral_kernel(const SpecArgs A) {
    const long long N = (long long)A.nx * A.ny * A.nz;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % A.nx);
        const long long r = q / A.nx;
        const int j = (int)(r % A.ny), k = (int)(r / A.ny);
        const int mi = i == 0 ? 0 : A.nx - i, mj = j == 0 ? 0 : A.ny - j, mk = k == 0 ? 0 : A.nz - k;
        const float2 zk = A.z[q];
        const float2 zm = A.z[((long long)mk * A.ny + mj) * A.nx + mi];
        // F^ = (Z_k + conj Z_-k)/2, G^ = (Z_k - conj Z_-k)/(2i)
        const float2 F = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 G = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        // P = conj(G) F * norm
        const float2 P = make_float2(A.norm * fmaf(G.x, F.x, G.y * F.y), A.norm * fmaf(G.x, F.y, -G.y * F.x));
        const float kx = wavenumber(i, A.nx, A.kx0), ky = wavenumber(j, A.ny, A.ky0), kz = wavenumber(k, A.nz, A.kz0);
        // -i k P = (k P.y, -k P.x); B1 = P + i(-i kx P), B2 = (-i ky P) + i(-i kz P); i (a + ib) = (-b, a)
        const float2 dx = make_float2(kx * P.y, -kx * P.x);
        const float2 dy = make_float2(ky * P.y, -ky * P.x);
        const float2 dz = make_float2(kz * P.y, -kz * P.x);
        A.b1[q] = make_float2(P.x - dx.y, P.y + dx.x);
        A.b2[q] = make_float2(dy.x - dz.y, dy.y + dz.x);
    }
}

__global__ void output_kernel(const float2* __restrict__ b1, const float2* __restrict__ b2, float4* ff, long long N,
                              int accumulate) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const float2 a = b1[q], b = b2[q];  // (E, Fx), (Fy, Fz)
        float4 v = make_float4(a.y, b.x, b.y, a.x);  // the spectra already hold -i k P: forces
        if (accumulate) {
            const float4 o = ff[q];
            v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
        }
        ff[q] = v;
    }
}

int ilog2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

cudaError_t fft_axis(float2* data, int n, int inner, int outer, float sign, cudaStream_t s) {
    if (n < 2) return cudaSuccess;
    const int L = inner == 1 ? (outer < kLines ? outer : kLines) : (inner < kLines ? inner : kLines);
    const size_t smem = (size_t)(n / 2 + L * n) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks, nbi = 1;
    if (inner == 1) {
        blocks = outer / L;  // outer = number of lines: a power of two, a multiple of L
    } else {
        nbi = inner / L;
        blocks = outer * nbi;
    }
    fft_pass_kernel<<<blocks, kFftThreads, smem, s>>>(data, n, ilog2i(n), inner, L, nbi, sign);
    return cudaGetLastError();
}

cudaError_t fft3(float2* data, int nx, int ny, int nz, float sign, cudaStream_t s) {
    cudaError_t e;
    if ((e = fft_axis(data, nx, 1, ny * nz, sign, s)) != cudaSuccess) return e;
    if ((e = fft_axis(data, ny, nx, nz, sign, s)) != cudaSuccess) return e;
    return fft_axis(data, nz, nx * ny, 1, sign, s);
}

}  // namespace

size_t fft_workspace_bytes(int nx, int ny, int nz) { return (size_t)3 * nx * ny * nz * sizeof(float2); }

cudaError_t launch_fft_correlate(const FftLaunch& L, cudaStream_t s) {
    const long long N = (long long)L.nx * L.ny * L.nz;
    float2* z = reinterpret_cast<float2*>(L.ws);
    float2* b1 = z + N;
    float2* b2 = b1 + N;
    const int threads = 256;
    const int blocks = (int)((N + threads - 1) / threads < 152LL * 16 ? (N + threads - 1) / threads : 152LL * 16);
    pack_kernel<<<blocks, threads, 0, s>>>(L.f, L.g, z, N, L.power);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = fft3(z, L.nx, L.ny, L.nz, -1.f, s)) != cudaSuccess) return e;
    SpecArgs A;
    A.z = z;
    A.b1 = b1;
    A.b2 = b2;
    A.nx = L.nx; A.ny = L.ny; A.nz = L.nz;
    A.kx0 = (float)(2.0 * kPi / (L.nx * (double)L.dx));
    A.ky0 = (float)(2.0 * kPi / (L.ny * (double)L.dy));
    A.kz0 = (float)(2.0 * kPi / (L.nz * (double)L.dz));
    A.norm = (float)((double)L.scale * (double)L.dx * L.dy * L.dz / (double)N);
    spectral_kernel<<<blocks, threads, 0, s>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = fft3(b1, L.nx, L.ny, L.nz, 1.f, s)) != cudaSuccess) return e;
    if ((e = fft3(b2, L.nx, L.ny, L.nz, 1.f, s)) != cudaSuccess) return e;
    output_kernel<<<blocks, threads, 0, s>>>(b1, b2, L.ff, N, L.accumulate);
    return cudaGetLastError();
}

}  // namespace pp
