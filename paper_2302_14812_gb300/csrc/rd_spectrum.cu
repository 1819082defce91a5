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

// The three components c0..c0+2 (E: c0 = 0, B: c0 = 3) of bin b of a cell's row, with vector loads.
template <typename T, int STRIDE>
struct Load3;
template <>
struct Load3<float, 8> {
    static __device__ __forceinline__ float3 get(const float* row, int b, int c0)
    {
        const float* v = row + (size_t)b * 8;
        const float4 a = __ldg(reinterpret_cast<const float4*>(v));
        if (c0 == 0) return make_float3(a.x, a.y, a.z);
        const float2 c = __ldg(reinterpret_cast<const float2*>(v + 4));
        return make_float3(a.w, c.x, c.y);
    }
};
template <>
struct Load3<double, 6> {
    static __device__ __forceinline__ float3 get(const double* row, int b, int c0)
    {
        const double* v = row + (size_t)b * 6;
        if (c0 == 0) {
            const double2 a = __ldg(reinterpret_cast<const double2*>(v));
            return make_float3((float)a.x, (float)a.y, (float)__ldg(v + 2));
        }
        const double2 c = __ldg(reinterpret_cast<const double2*>(v + 4));
        return make_float3((float)__ldg(v + 3), (float)c.x, (float)c.y);
    }
};

// Shared-memory index of element i of a transform: one float2 of padding after every 32, so that
// the bit-reversed stores of the load phase (consecutive bins -> elements N/32 apart) spread over
// the banks.
__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

__device__ __forceinline__ void butterfly(float2* z, int i0, int i1, float2 w)
{
    const float2 a = z[pad(i0)], b = cmul(z[pad(i1)], w);
    z[pad(i0)] = make_float2(a.x + b.x, a.y + b.y);
    z[pad(i1)] = make_float2(a.x - b.x, a.y - b.y);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// Two stages at once on the four elements i0 + {0, h, 2h, 3h} (i0 = 4 G h + p, p < h): span h
// pairs (0, 1) and (2, 3) with twiddle w1 = exp(-2 pi i p / (2h)), then span 2h pairs (0, 2) with
// w2a = exp(-2 pi i p / (4h)) and (1, 3) with w2b = exp(-2 pi i (p + h) / (4h)).
__device__ __forceinline__ void butterfly2x2(float2* z, int i0, int h, float2 w1, float2 w2a, float2 w2b)
{
    const float2 a0 = z[pad(i0)], a1 = cmul(z[pad(i0 + h)], w1);
    const float2 a2 = z[pad(i0 + 2 * h)], a3 = cmul(z[pad(i0 + 3 * h)], w1);
    const float2 b0 = cadd(a0, a1), b1 = csub(a0, a1), b2 = cmul(cadd(a2, a3), w2a), b3 = cmul(csub(a2, a3), w2b);
    z[pad(i0)] = cadd(b0, b2);
    z[pad(i0 + 2 * h)] = csub(b0, b2);
    z[pad(i0 + h)] = cadd(b1, b3);
    z[pad(i0 + 3 * h)] = csub(b1, b3);
}

// One CTA per cell at a time (persistent over cells).  Shared memory: Z1 and Z2 (N elements each,
// padded) and the twiddles of every stage, stage h (span h) holding exp(-2 pi i p / (2h)), p < h,
// at h - 1 + p (contiguous in p, so a warp's lanes read consecutive entries).  The bins are loaded
// in bit-reversed order, so in-place decimation-in-time butterflies leave the transforms in
// natural order.
template <typename T, int STRIDE>
__global__ void __launch_bounds__(256) k_spectrum_fused(const T* __restrict__ fields, int n_pix, int N, int logN,
                                                        int c0, const float2* __restrict__ tw_g, float scale,
                                                        float* __restrict__ P)
{
    extern __shared__ float2 sm[];
    const int zlen = pad(N - 1) + 1;
    float2* z1 = sm;
    float2* z2 = sm + zlen;
    float2* tw = sm + 2 * zlen;
    const int half_n = N >> 1;
    for (int h = 1; h < N; h <<= 1) {
        const int step = half_n / h;
        for (int p = threadIdx.x; p < h; p += blockDim.x) tw[h - 1 + p] = tw_g[p * step];
    }
    const int nk = half_n + 1;
    for (int cell = blockIdx.x; cell < n_pix; cell += gridDim.x) {
        const T* row = fields + (size_t)cell * N * STRIDE;
#pragma unroll 4
        for (int b = threadIdx.x; b < N; b += blockDim.x) {
            const int r = pad((int)(__brev((unsigned)b) >> (32 - logN)));
            const float3 v = Load3<T, STRIDE>::get(row, b, c0);
            z1[r] = make_float2(v.x, v.y);
            z2[r] = make_float2(v.z, 0.f);
        }
        __syncthreads();
        int h = 1;
        for (; 4 * h <= N; h <<= 2) {                 // stages of span h and 2h in one pass
            const float2* wa = tw + (h - 1);
            const float2* wb = tw + (2 * h - 1);
            for (int t = threadIdx.x; t < (N >> 2); t += blockDim.x) {
                const int G = t / h, p = t - G * h;
                const int i0 = 4 * G * h + p;
                const float2 w1 = wa[p], w2a = wb[p], w2b = wb[p + h];
                butterfly2x2(z1, i0, h, w1, w2a, w2b);
                butterfly2x2(z2, i0, h, w1, w2a, w2b);
            }
            __syncthreads();
        }
        if (h < N) {                                  // odd number of stages: the last, span N/2
            const float2* wh = tw + (h - 1);
            for (int t = threadIdx.x; t < half_n; t += blockDim.x) {
                const float2 w = wh[t];
                butterfly(z1, t, t + h, w);
                butterfly(z2, t, t + h, w);
            }
            __syncthreads();
        }
        float* out = P + (size_t)cell * nk;
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            const int km = (N - k) & (N - 1);
            const float2 a = z1[pad(k)], am = z1[pad(km)], c = z2[pad(k)];
            const float pxy = 0.5f * (a.x * a.x + a.y * a.y + am.x * am.x + am.y * am.y);
            out[k] = scale * (pxy + (c.x * c.x + c.y * c.y));
        }
        __syncthreads();
    }
}

int grid_for(long long n, int threads) { return grid_stride_blocks(n, threads, 32); }

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
        const size_t smem = sizeof(float2) * (2 * (size_t)(N + N / 32) + N);
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
