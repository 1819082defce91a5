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

// Shared-memory index of element i of a transform: one float2 of padding after every 16, so that
// the strided reads and writes of every radix-16 pass (and of the shorter last pass) fall on
// distinct banks.
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// exp(-2 pi i j / 16), j = 0..7: the roots the in-register transforms of length <= 16 multiply by
__device__ __forceinline__ float2 root16(int j)
{
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
    const float re[8] = {1.f, c1, h, s1, 0.f, -s1, -h, -c1};
    const float im[8] = {0.f, -s1, -h, -c1, -1.f, -c1, -h, -s1};
    return make_float2(re[j], im[j]);
}

// a * exp(-2 pi i j / 16) with the trivial roots (1, -i) taken without a multiply; j is a
// compile-time constant after unrolling
__device__ __forceinline__ float2 mul_root16(float2 a, int j)
{
    if (j == 0) return a;
    if (j == 4) return make_float2(a.y, -a.x);
    return cmul(a, root16(j));
}

// In-register DFT of length R (2, 4, 8, 16): X[k] = sum_r a[r] exp(-2 pi i r k / R), by radix-2
// decimation in frequency; the result is left in bit-reversed order (a[bitrev(k)] = X[k]).
template <int R>
constexpr int log2_of() { return R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1; }

template <int R>
__device__ __forceinline__ void dft_bitrev(float2 (&a)[R])
{
    constexpr int L = log2_of<R>();
#pragma unroll
    for (int st = 0; st < L; ++st) {
        const int h = R >> (st + 1);                            // span of this stage
#pragma unroll
        for (int g = 0; g < (1 << st); ++g) {
#pragma unroll
            for (int i = 0; i < R / (2 << st); ++i) {
                const int j = g * (R >> st);
                const float2 u = a[j + i], v = a[j + i + h];
                a[j + i] = cadd(u, v);
                a[j + i + h] = mul_root16(csub(u, v), i * (8 / h));     // exp(-2 pi i i / (2h))
            }
        }
    }
}

template <int R>
__device__ __forceinline__ constexpr int bitrev(int k)
{
    constexpr int L = log2_of<R>();
    int r = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) r |= ((k >> i) & 1) << (L - 1 - i);
    return r;
}

// exp(-2 pi i j / N) for 0 <= j < N from the half-circle table tw[j] (j < N/2, in shared memory)
__device__ __forceinline__ float2 twiddle(const float2* tw, int j, int half_n)
{
    if (j < half_n) return tw[j];
    const float2 w = tw[j - half_n];
    return make_float2(-w.x, -w.y);
}

// One Stockham pass of radix R on both transforms of a cell (in place in shared memory, or reading
// the cell's bins from global memory when s = 1 and G): with n = N / s and m = n / R, butterfly
// (p, q), p < m, q < s, takes a_r = x[q + s (p + r m)], r < R, forms b_k = DFT_R(a)[k] and writes
// y[q + s (R p + k)] = b_k exp(-2 pi i p k / n).  After the passes of radices R1 R2 ... = N the
// transform is in natural order.  Each thread holds 16 elements of each transform (16 / R
// butterflies); all reads of a pass finish before its writes.
template <int R, bool G, typename T, int STRIDE>
__device__ __forceinline__ void spec_pass(float2* z1, float2* z2, const T* row, int c0, int N, int s,
                                          const float2* tw, int tid)
{
    constexpr int NB = 16 / R;                  // butterflies per thread
    const int n = N / s, m = n / R;
    const int nb = N / R;                       // butterflies per transform
    float2 a1[NB][R], a2[NB][R];
    int bq[NB], bp[NB];
    bool on[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int t = tid + u * blockDim.x;
        on[u] = t < nb;
        bq[u] = t % s;
        bp[u] = t / s;
        if (on[u]) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = bq[u] + s * (bp[u] + r * m);
                if (G) {
                    const float3 v = Load3<T, STRIDE>::get(row, i, c0);
                    a1[u][r] = make_float2(v.x, v.y);
                    a2[u][r] = make_float2(v.z, 0.f);
                } else {
                    a1[u][r] = z1[pad(i)];
                    a2[u][r] = z2[pad(i)];
                }
            }
        }
    }
    __syncthreads();    // every read of the pass is done (first pass: the twiddle table is filled)
    const int half_n = N >> 1;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        if (!on[u]) continue;
        dft_bitrev<R>(a1[u]);
        dft_bitrev<R>(a2[u]);
        const int o = bq[u] + s * R * bp[u];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            float2 b1 = a1[u][bitrev<R>(k)], b2 = a2[u][bitrev<R>(k)];
            if (k > 0) {
                const float2 w = twiddle(tw, bp[u] * k * s, half_n);      // exp(-2 pi i p k / n)
                b1 = cmul(b1, w);
                b2 = cmul(b2, w);
            }
            z1[pad(o + s * k)] = b1;
            z2[pad(o + s * k)] = b2;
        }
    }
    __syncthreads();
}

// The passes after the first, at stride S, of a length-N transform: radix 16 while 16 elements
// remain per butterfly, then the remaining radix (a compile-time sequence, so that every pass's
// registers are allocated on their own).
template <int N, int S, typename T, int STRIDE>
__device__ __forceinline__ void spec_passes(float2* z1, float2* z2, const float2* tw, int tid)
{
    if constexpr (S < N) {
        constexpr int R = N / S >= 16 ? 16 : N / S;
        spec_pass<R, false, T, STRIDE>(z1, z2, nullptr, 0, N, S, tw, tid);
        spec_passes<N, S * R, T, STRIDE>(z1, z2, tw, tid);
    }
}

constexpr int spec_threads(int N) { return N / 16 > 128 ? N / 16 : 128; }
// resident CTAs per SM the kernel is compiled for: 512 threads per SM (128 registers a thread)
constexpr int spec_min_blocks(int N) { return 512 / spec_threads(N); }

// One CTA per cell, spec_threads(N) threads.  Shared memory: Z1 and Z2 (N elements each, padded)
// and the N/2 twiddles.  The first pass reads the cell's bins from global memory (consecutive
// threads, consecutive bins); the power of frequency k needs Z1 at k and N - k, so it is formed
// from shared memory after the last pass.  (A CTA looping over cells keeps every pass's state
// live across the loop and spills; a fresh CTA per cell fits the registers, and reloading the
// twiddles from L2 costs N/2 x 8 bytes per cell.)
template <int N, typename T, int STRIDE>
__global__ void __launch_bounds__(spec_threads(N), spec_min_blocks(N)) k_spectrum_fused(const T* __restrict__ fields,
                                                                                        int c0,
                                                                                        const float2* __restrict__ tw_g,
                                                                                        float scale, float* __restrict__ P)
{
    extern __shared__ float2 sm[];
    constexpr int zlen = N + N / 16;
    constexpr int R1 = N >= 16 ? 16 : N;
    float2* z1 = sm;
    float2* z2 = sm + zlen;
    float2* tw = sm + 2 * zlen;
    const int tid = threadIdx.x;
    const size_t cell = blockIdx.x;
    const T* row = fields + cell * N * STRIDE;
    // filled before the first pass's barrier, read after it
    for (int j = tid; j < N / 2; j += blockDim.x) tw[j] = tw_g[j];
    spec_pass<R1, true, T, STRIDE>(z1, z2, row, c0, N, 1, tw, tid);
    spec_passes<N, R1, T, STRIDE>(z1, z2, tw, tid);
    constexpr int nk = N / 2 + 1;
    float* out = P + cell * nk;
    for (int k = tid; k < nk; k += blockDim.x) {
        const int km = (N - k) & (N - 1);
        const float2 a = z1[pad(k)], am = z1[pad(km)], c = z2[pad(k)];
        const float pxy = 0.5f * (a.x * a.x + a.y * a.y + am.x * am.x + am.y * am.y);
        out[k] = scale * (pxy + (c.x * c.x + c.y * c.y));
    }
}

template <int N, typename T, int STRIDE>
cudaError_t launch_fused_n(const T* fields, int n_pix, int c0, const float2* tw, float scale, float* P,
                           cudaStream_t s)
{
    constexpr int threads = spec_threads(N);
    const size_t smem = sizeof(float2) * (2 * (size_t)(N + N / 16) + N / 2);
    auto k = k_spectrum_fused<N, T, STRIDE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<n_pix, threads, smem, s>>>(fields, c0, tw, scale, P);
    return cudaGetLastError();
}

template <typename T, int STRIDE>
cudaError_t launch_fused(const T* fields, int n_pix, int N, int c0, const float2* tw, float scale, float* P,
                         cudaStream_t s)
{
    switch (N) {
    case 2: return launch_fused_n<2, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 4: return launch_fused_n<4, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 8: return launch_fused_n<8, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 16: return launch_fused_n<16, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 32: return launch_fused_n<32, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 64: return launch_fused_n<64, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 128: return launch_fused_n<128, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 256: return launch_fused_n<256, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 512: return launch_fused_n<512, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 1024: return launch_fused_n<1024, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 2048: return launch_fused_n<2048, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 4096: return launch_fused_n<4096, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    case 8192: return launch_fused_n<8192, T, STRIDE>(fields, n_pix, c0, tw, scale, P, s);
    default: return cudaErrorInvalidValue;
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
        if (precision == RD_MIXED)
            return launch_fused<float, 8>(static_cast<const float*>(fields), n_pix, N, c0, tw, scale, P, s);
        return launch_fused<double, 6>(static_cast<const double*>(fields), n_pix, N, c0, tw, scale, P, s);
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
