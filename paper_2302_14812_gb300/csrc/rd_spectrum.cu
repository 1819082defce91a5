// Power spectra of the detector's time series (Section 4: the detector data are Fourier
// transformed in time and compared with the synchrotron spectra, Eq. 8 and Eq. 9).
//
// For every cell j and frequency index k = 0..N/2 (N = n_bins, a power of two):
//     P[j][k] = dt_det^2 * sum_c | sum_b F_c[j][b] exp(-2 pi i k b / N) |^2
// with F = E or B.  Two complex transforms per cell carry the three real components:
// Z1 = F_x + i F_y gives |Fx(k)|^2 + |Fy(k)|^2 = (|Z1(k)|^2 + |Z1(N-k)|^2) / 2, and Z2 = F_z gives
// |Fz(k)|^2 = |Z2(k)|^2.  Twiddles exp(-2 pi i j / N) are computed in FP64 once per length.
// N <= kFusedMaxN: one kernel reads a cell's bins, runs both FP32 radix-2 transforms in shared
// memory and writes the cell's spectrum (the fields are read once, the spectrum written once).
// Longer series: FP32 Stockham radix-2 passes over the whole batch, one launch per pass.
#include <math.h>

#include <algorithm>

#include "rd_internal.cuh"

namespace rd {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Z[2 j][b] = F_x + i F_y,  Z[2 j + 1][b] = F_z + 0 i  (component offset c0 = 0 for E, 3 for B)
template <typename T, int STRIDE>
__global__ void k_pack_spectrum_input(const T* __restrict__ fields, int n_pix, int n_bins, int c0,
                                      float2* __restrict__ z)
{
    const long long total = (long long)n_pix * n_bins;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = i / n_bins, b = i - j * n_bins;
        const T* f = fields + i * STRIDE + c0;
        z[(2 * j) * n_bins + b] = make_float2((float)f[0], (float)f[1]);
        z[(2 * j + 1) * n_bins + b] = make_float2((float)f[2], 0.f);
    }
}

// One Stockham pass (n = N / s, s = 2^stage) over `batch` transforms of length N:
//   a = x[q + s p], b = x[q + s (p + n/2)],  y[q + s 2p] = a + b,  y[q + s (2p + 1)] = (a - b) w^p,
// w = exp(-2 pi i / n), p < n/2, q < s; w^p = tw[p s] with tw[j] = exp(-2 pi i j / N).
__global__ void k_fft_pass(const float2* __restrict__ x, float2* __restrict__ y, int N, int s,
                           const float2* __restrict__ tw, long long batch)
{
    const int half = N >> 1;
    const long long total = batch * half;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long bt = t / half;
        const int i = (int)(t - bt * half);          // i = p s + q
        const int q = i & (s - 1);
        const int p = i / s;
        const float2* xb = x + bt * N;
        float2* yb = y + bt * N;
        const float2 a = xb[i], b = xb[i + half];
        const float2 w = tw[p * s];
        yb[q + 2 * s * p] = make_float2(a.x + b.x, a.y + b.y);
        yb[q + 2 * s * p + s] = cmul(make_float2(a.x - b.x, a.y - b.y), w);
    }
}

__global__ void k_spectrum_power(const float2* __restrict__ X, int n_pix, int N, float scale,
                                 float* __restrict__ P)
{
    const int nk = N / 2 + 1;
    const long long total = (long long)n_pix * nk;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = i / nk;
        const int k = (int)(i - j * nk);
        const int km = (N - k) & (N - 1);
        const float2 z1 = X[(2 * j) * N + k], z1m = X[(2 * j) * N + km], z2 = X[(2 * j + 1) * N + k];
        const float pxy = 0.5f * (z1.x * z1.x + z1.y * z1.y + z1m.x * z1m.x + z1m.y * z1m.y);
        const float pz = z2.x * z2.x + z2.y * z2.y;
        P[i] = scale * (pxy + pz);
    }
}

__device__ __forceinline__ void butterfly(float2* z, int i0, int i1, float2 w)
{
    const float2 a = z[i0], b = cmul(z[i1], w);
    z[i0] = make_float2(a.x + b.x, a.y + b.y);
    z[i1] = make_float2(a.x - b.x, a.y - b.y);
}

// One CTA per cell at a time (persistent over cells).  Shared memory: Z1[N], Z2[N], twiddles[N/2].
// The bins are loaded in bit-reversed order, so in-place decimation-in-time butterflies (span h,
// twiddle exp(-2 pi i p / (2h)) = tw[p N / (2h)]) leave the transforms in natural order.
template <typename T, int STRIDE>
__global__ void __launch_bounds__(256) k_spectrum_fused(const T* __restrict__ fields, int n_pix, int N, int logN,
                                                        int c0, const float2* __restrict__ tw_g, float scale,
                                                        float* __restrict__ P)
{
    extern __shared__ float2 sm[];
    float2* z1 = sm;
    float2* z2 = sm + N;
    float2* tw = sm + 2 * N;
    const int half_n = N >> 1;
    for (int j = threadIdx.x; j < half_n; j += blockDim.x) tw[j] = tw_g[j];
    const int nk = half_n + 1;
    for (int cell = blockIdx.x; cell < n_pix; cell += gridDim.x) {
        const T* f = fields + (size_t)cell * N * STRIDE + c0;
        for (int b = threadIdx.x; b < N; b += blockDim.x) {
            const int r = (int)(__brev((unsigned)b) >> (32 - logN));
            const T* v = f + (size_t)b * STRIDE;
            z1[r] = make_float2((float)v[0], (float)v[1]);
            z2[r] = make_float2((float)v[2], 0.f);
        }
        __syncthreads();
        for (int h = 1; h < N; h <<= 1) {
            const int step = half_n / h;
            for (int t = threadIdx.x; t < half_n; t += blockDim.x) {
                const int g = t / h, p = t - g * h;
                const int i0 = 2 * g * h + p;
                const float2 w = tw[p * step];
                butterfly(z1, i0, i0 + h, w);
                butterfly(z2, i0, i0 + h, w);
            }
            __syncthreads();
        }
        float* out = P + (size_t)cell * nk;
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            const int km = (N - k) & (N - 1);
            const float2 a = z1[k], am = z1[km], c = z2[k];
            const float pxy = 0.5f * (a.x * a.x + a.y * a.y + am.x * am.x + am.y * am.y);
            out[k] = scale * (pxy + (c.x * c.x + c.y * c.y));
        }
        __syncthreads();
    }
}

int grid_for(long long n, int threads)
{
    long long g = (n + threads - 1) / threads;
    if (g > 152LL * 32) g = 152LL * 32;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

void fill_twiddles(float2* host, int N)
{
    const double two_pi = 6.283185307179586476925287;
    for (int j = 0; j < N / 2; ++j) {
        const double a = -two_pi * (double)j / (double)N;
        host[j] = make_float2((float)cos(a), (float)sin(a));
    }
}

bool spectrum_fused(int N) { return N >= 2 && N <= kFusedMaxN; }

// z: [2 n_pix][N] work array, y: same size (unused for N <= kFusedMaxN); tw: [N/2].
cudaError_t launch_power_spectrum(const void* fields, int precision, int n_pix, int N, int c0, float2* z,
                                  float2* y, const float2* tw, float scale, float* P, cudaStream_t s)
{
    if (spectrum_fused(N)) {
        int logN = 0;
        while ((1 << logN) < N) ++logN;
        const size_t smem = sizeof(float2) * (2 * (size_t)N + N / 2);
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e;
        if (precision == RD_MIXED) {
            auto k = k_spectrum_fused<float, 8>;
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem);
            if (e != cudaSuccess) return e;
            const int grid = (int)std::min<long long>(n_pix, (long long)sms * std::max(1, per_sm));
            k<<<grid, 256, smem, s>>>(static_cast<const float*>(fields), n_pix, N, logN, c0, tw, scale, P);
        } else {
            auto k = k_spectrum_fused<double, 6>;
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem);
            if (e != cudaSuccess) return e;
            const int grid = (int)std::min<long long>(n_pix, (long long)sms * std::max(1, per_sm));
            k<<<grid, 256, smem, s>>>(static_cast<const double*>(fields), n_pix, N, logN, c0, tw, scale, P);
        }
        return cudaGetLastError();
    }
    const long long n = (long long)n_pix * N;
    if (precision == RD_MIXED)
        k_pack_spectrum_input<float, 8><<<grid_for(n, 256), 256, 0, s>>>(static_cast<const float*>(fields), n_pix,
                                                                          N, c0, z);
    else
        k_pack_spectrum_input<double, 6><<<grid_for(n, 256), 256, 0, s>>>(static_cast<const double*>(fields),
                                                                           n_pix, N, c0, z);
    cudaError_t e = cudaGetLastError();
    float2* a = z;
    float2* b = y;
    const long long batch = 2LL * n_pix;
    for (int st = 1; st < N && e == cudaSuccess; st <<= 1) {
        k_fft_pass<<<grid_for(batch * (N / 2), 256), 256, 0, s>>>(a, b, N, st, tw, batch);
        e = cudaGetLastError();
        float2* t = a;
        a = b;
        b = t;
    }
    if (e != cudaSuccess) return e;
    const long long np = (long long)n_pix * (N / 2 + 1);
    k_spectrum_power<<<grid_for(np, 256), 256, 0, s>>>(a, n_pix, N, scale, P);
    return cudaGetLastError();
}

}  // namespace rd
