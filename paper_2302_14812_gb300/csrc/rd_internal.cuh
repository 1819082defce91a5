// Internal declarations of the radiation-deposit library (sm_103a).
//
// Data layout in device memory
//   cell table     D4     [n_pix]              (x, y, z, T0 = t_min + pix_t0)
//   mixed fields   float   [n_pix][n_bins][8]  (Ex Ey Ez Bx | By Bz 0 0): one 32-byte sector per bin
//   fp64 fields    double  [n_pix][n_bins][6]  (Ex Ey Ez Bx By Bz)
//   records        RecS / RecD [n_part][n_samples]: per-sample quantities of Algorithm 1,
//                  computed once per call and read by every cell (staged through shared memory
//                  with bulk asynchronous copies).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>

#include "../../include/rd.h"

namespace rd {

// ---------------------------------------------------------------------------------------------
// error bits latched on the device (bit i = 1 << rd_status value)
// ---------------------------------------------------------------------------------------------
enum : unsigned {
    ERRBIT_TIMEOUT = 1u << RD_ERR_TIMEOUT,
    ERRBIT_BOUNDS = 1u << RD_ERR_BOUNDS,
    ERRBIT_INPUT = 1u << RD_ERR_INPUT,
};

struct DevCounters {
    unsigned errors;
    unsigned pad;
    unsigned long long clipped;
    unsigned long long crossings;   // bin edges crossed by arrival intervals (mixed path)
};

// ---------------------------------------------------------------------------------------------
// per-sample records
// ---------------------------------------------------------------------------------------------
// Mixed path, per-sample constants of interval k (16 values), with signs chosen so that every step
// of the field is an add / mul / fma:
//   nx, ny, nz = -x_k               nhig2 = -gamma_k^-2 / 2
//   nbx..nbz   = -beta_k            ig2n  = Q (near ? gamma_k^-2 : 0)
//   bdx..bdz   = Q (far ? betadot_k : 0)             dtg = dt g_k,  g_k = 1 - |vbar_k|^2
//   d2x..d2z   = 2 (beta_k - vbar_k)  gd  = g_k + |beta_k - vbar_k|^2
// (vbar_k = (x_k - x_{k-1})/dt is the chord velocity of the interval).  Q = -q_p dt/dt_det in the
// records of a deposit (charge and bin-weight scale folded in: E' and d x E' come out scaled by
// Q), Q = 1 in the records of the adjoint.
struct __align__(16) RecS {
    float nx, ny, nz, nhig2;
    float nbx, nby, nbz, ig2n;
    float bdx, bdy, bdz, dtg;
    float d2x, d2y, d2z, gd;
};
static_assert(sizeof(RecS) == 64, "RecS must be 64 bytes");

struct __align__(32) D4 {
    double x, y, z, w;
};

// FP64 path, 96 bytes: (x_k, t_k), (beta_k, q gamma_k^-2), (q betadot_k, 0), with t_k = t0 + k dt rounded
// as Eq. 2's arrival time takes it and q the particle's charge; gamma^-2 is stored as zero without the
// velocity term (RD_NEAR) and betadot as zero without the acceleration term (RD_FAR).  The FP64 adjoint
// takes the records with q = 1 and both terms.
struct __align__(32) RecD {
    D4 xa;
    D4 bb;
    D4 bd;
};
static_assert(sizeof(RecD) == 96, "RecD must be 96 bytes");

// ---------------------------------------------------------------------------------------------
// kernel parameter blocks
// ---------------------------------------------------------------------------------------------
struct DepositParams {
    const void* rec;            // RecS or RecD [n_part][n_samples]
    const double* x;            // [n_part][n_samples][3] FP64 positions (anchors of the mixed path)
    const double* q;            // [n_part] or null
    const D4* cells;            // [n_pix] (x, y, z, T0)
    void* fields;               // float [n_pix][n_bins][8] or double [n_pix][n_bins][6]
    DevCounters* counters;
    int n_pix;
    int n_bins;
    int n_samples;              // S + 1
    int n_part;
    int chunk;                  // intervals per work item
    int k_first;                // first interval deposited (1, or 2 for a streamed call that carries
                                // two earlier samples)
    int n_chunks;               // ceil(S / chunk)
    int n_cell_blocks;          // ceil(n_pix / cells per CTA)
    float W;                    // mixed: bin width in units of dt (dt_det / dt)
    float invW;
    double t0;
    double dt;
    double inv_dt_det;
    float dt_f;
    float du_scale;             // dt / dt_det
    int ff;                     // far-field limit (RD_FARFIELD): Eq. 3, radiation term at (n_c, R_c)
    int lin;                    // 0: held field; 1: linear in arrival time (RD_LINEAR); 2: the previous
                                // sample's field held (RD_HOLD_PREV); 3: quadratic in arrival time
                                // (RD_QUADRATIC); 1-3 carry the previous field, 3 the one before too
    int k_real0 = 0;            // index in the whole trajectory of this call's sample 0 (streamed calls)
    int group = 1;              // mixed kernel work order: cell blocks per group (cell_group)
    int cpc = 256;              // mixed kernel shape: cells per CTA (64, 128, 256) ...
    int nc = 2;                 // ... and cells per thread (1, 2); n_cell_blocks counts blocks of cpc cells
};

#ifdef __CUDACC__
// Work item (particle p, cell block cb, step chunk ch) of linear index idx for the mixed kernels:
// chunks slowest; inside a chunk, groups of P.group cell blocks; inside a group the cell block
// fastest, then the particle.  Consecutive CTAs so take one particle to the group's cell blocks
// back to back (its staged records are read from DRAM once per group, then from L2) while the
// resident CTAs reduce into the group's detector slice.  Odd groups take the particles in reverse
// order, so that a group starts on the records the previous one read last (still in L2).
// group = 1 is particle-fastest order.
__device__ __forceinline__ void item_coords(unsigned idx, const DepositParams& P, int& p, int& cb, int& ch)
{
    // 32-bit arithmetic: a launch (or a batch segment) holds fewer than 2^31 items (host-checked)
    const unsigned per_chunk = (unsigned)P.n_cell_blocks * (unsigned)P.n_part;
    ch = (int)(idx / per_chunk);
    unsigned r = idx - (unsigned)ch * per_chunk;
    const unsigned G = (unsigned)P.group;
    const unsigned per_group = G * (unsigned)P.n_part;
    const unsigned g = r / per_group;
    r -= g * per_group;
    const unsigned Gg = min(G, (unsigned)P.n_cell_blocks - g * G);
    cb = (int)(g * G + r % Gg);
    p = (int)(r / Gg);
    if (g & 1u) p = P.n_part - 1 - p;
}
#endif

constexpr int kDepositThreads = 256;   // FP64 kernel: one cell per thread
#ifndef RD_MIXED_MINBLOCKS
#define RD_MIXED_MINBLOCKS (RD_MIXED_CELLS >= 4 ? 6 : 5)
#endif
#ifndef RD_MIXED_CELLS
#define RD_MIXED_CELLS 2
#endif
constexpr int kMixedCells = RD_MIXED_CELLS;    // mixed kernel: cells walked by one thread
constexpr int kMixedCellsPerCta = 256;
constexpr int kMixedThreads = kMixedCellsPerCta / kMixedCells;
constexpr int kMixedMaxBins = 1 << 22;         // bins per cell of an RD_MIXED detector
#ifndef RD_TILE_STEPS
#define RD_TILE_STEPS 64
#endif
constexpr int kTileSteps = RD_TILE_STEPS;   // intervals per shared-memory tile
constexpr int kDefaultChunk = 2048;    // intervals per work item (one FP64 anchor at each end)
constexpr int kBatchItemsPerSm = 512;  // work items per multiprocessor the batched deposit aims for
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // give up a wait after 2 s

// host helpers (rd_api.cu)
int sm_count();    // multiprocessors of the current device (queried once per device)
// CTAs of a grid-stride kernel over n items: enough for n at `threads` per CTA, at most per_sm
// CTAs per multiprocessor of the current device, at least one
int grid_stride_blocks(long long n, int threads, int per_sm);
// Default intervals per work item of the deposit kernels: kDefaultChunk (at most S), halved while
// the grid (cell blocks x particles x chunks) would hold fewer than 8 CTAs per multiprocessor.
int auto_chunk(long long n_cell_blocks, long long n_part, int S);
// Cell blocks per group of the mixed kernels' work order (item_coords): as many as keep the group's
// active detector slice (cells_per_cta x 32 bytes x the bins a step chunk of `chunk` of the
// trajectory's n_intervals spans, per block) within RD_GROUP_SLICE_MB, at most 8.
int cell_group(int n_cell_blocks, int n_bins, int cells_per_cta, int chunk, int n_intervals);
// Deposit-shape tuning cache (rd_tune.cu): entries keyed by device and problem, in a JSON file.
struct TuneEntry {
    int cpc, nc, chunk, group;
    double ms;
};
bool tune_cache_load(const char* path, std::map<std::string, TuneEntry>& out, std::string& err);
bool tune_cache_store(const char* path, const std::string& key, const TuneEntry& e, std::string& err);
// Check of a detector's `flags` (include/rd.h): null if valid, else the reason.
const char* flags_error(int flags);

// launchers (rd_deposit.cu)
// qscale != 0: deposit records, betadot and gamma^-2 terms multiplied by -q_p * qscale (q null:
// unit charges); qscale == 0: plain records (adjoint).
cudaError_t launch_precompute_mixed(const double* x, const double* u, const double* q, double qscale, int n_part,
                                    int n_samples, double dt, int flags, RecS* rec, DevCounters* counters,
                                    cudaStream_t s);
cudaError_t launch_precompute_fp64(const double* x, const double* u, const double* q, int n_part, int n_samples,
                                   double t0, double dt, int flags, RecD* rec, DevCounters* counters, cudaStream_t s);
cudaError_t launch_deposit_mixed(const DepositParams& p, cudaStream_t s);
// shapes of the mixed kernel compiled into the library (held field, exact Eq. 1; the far-field and
// interpolation variants and the batch kernel run the default shape, kMixedCellsPerCta x kMixedCells)
bool mixed_shape_supported(int cells_per_cta, int cells_per_thread);
cudaError_t launch_deposit_batch(int family, const DepositParams* probs, const long long* item_off, int n_probs,
                                 unsigned long long* next_item, cudaStream_t s);
// resident CTAs of the persistent batch kernel of a walk family (4 x far field + 0 held / 1 linear
// family / 2 quadratic) on the current device
int batch_grid(int family);
cudaError_t launch_deposit_fp64(const DepositParams& p, int flags, cudaStream_t s);
// adjoint (rd_adjoint.cu)
struct AdjointParams {
    const RecS* rec;            // [n_part][n_samples] (mixed kernel)
    const RecD* recd;           // [n_part][n_samples] (FP64 kernel)
    const double* x;            // [n_part][n_samples][3] FP64 positions (anchors)
    const double* q;            // [n_part] or null
    const D4* cells;            // [n_pix]
    const float* seed;          // [n_pix][n_bins][8] upstream gradient (E xyz, B xyz) in field layout
                                // (compensated kernel: [n_pix][n_bins][16], double-float)
    const double* seedd;        // [n_pix][n_bins][6] the same in FP64 (FP64 kernel)
    double* gx;                 // [n_part][n_samples][3] += d loss / d x
    double* gbeta;              // [n_part][n_samples][3] += d loss / d beta (scratch, FP64)
    const void* recc;           // compensated kernel: double-float records [n_part][n_samples]
    double* gu;                 // compensated kernel: [n_part][n_samples][3] += d loss / d u
    DevCounters* counters;
    int n_pix, n_bins, n_samples, n_part, chunk, n_chunks, n_cell_blocks;
    int flags;
    double t0, dt, inv_dt_det;
    float dt_f, du_scale, W, invW;
    float inv_dt_det_f, inv_dt_f;   // 1/dt_det and 1/dt in FP32 (no conversion or division per step)
    float edge_tol;             // mixed: distance (dt units) from a bin edge below which an arrival's bin
                                // is taken from Eq. 2 in FP64 for its end-point terms
};
#ifndef RD_ADJ_THREADS
#define RD_ADJ_THREADS 128
#endif
#ifndef RD_ADJ_CELLS
#define RD_ADJ_CELLS 1
#endif
#ifndef RD_ADJ_MINBLOCKS
#define RD_ADJ_MINBLOCKS (RD_ADJ_CELLS == 1 ? 6 : 4)
#endif
constexpr int kAdjointThreads = RD_ADJ_THREADS;
constexpr int kAdjointCells = RD_ADJ_CELLS;       // cells per thread
constexpr int kAdjointCellsPerCta = kAdjointThreads * kAdjointCells;
cudaError_t launch_pack_seed(const void* gE, const void* gB, int dtype, int n_pix, int n_bins, float* seed,
                             cudaStream_t s);
cudaError_t launch_adjoint_mixed(const AdjointParams& p, cudaStream_t s);
cudaError_t launch_pack_seed64(const void* gE, const void* gB, int dtype, int n_pix, int n_bins, double* seed,
                               cudaStream_t s);
cudaError_t launch_adjoint_fp64(const AdjointParams& p, cudaStream_t s);
constexpr int kAdjointFp64Threads = 128;   // FP64 adjoint: one cell per thread
// compensated (double-float) adjoint of the mixed deposit (rd_adjoint_comp.cu)
constexpr int kAdjointCompThreads = 128;   // one cell per thread
size_t comp_record_bytes();                // bytes of one per-sample record
// upstream gradient as double-float seed rows [n_pix][n_bins][16] floats (64 bytes per bin)
cudaError_t launch_pack_seed_df(const void* gE, const void* gB, int dtype, int n_pix, int n_bins, float* seed,
                                cudaStream_t s);
cudaError_t launch_precompute_comp(const double* x, const double* u, int n_part, int n_samples, double dt, int flags,
                                   void* rec, DevCounters* counters, cudaStream_t s);
cudaError_t launch_adjoint_comp(const AdjointParams& p, cudaStream_t s);
cudaError_t launch_gbeta_to_gu(const double* u, const double* gbeta, double* gu, long long n_samples_total,
                               cudaStream_t s);

// run-time coupling (rd_push.cu): Boris steps in a uniform magnetic field B[3] (host array)
cudaError_t launch_push_boris(int n_part, int n_steps, double dt, const double* B, double qm, double* x, double* u,
                              double* x_out, double* u_out, cudaStream_t s);
// diagnostics (rd_diag.cu): FMA throughput of the current device in TFLOP/s (one FMA = 2 flops), and one
// CTA whose bounded wait on an mbarrier phase that nothing completes runs out after limit_ns (the
// expiry is recorded in *errors as the kernels record it)
cudaError_t measure_fma_peaks(cudaStream_t s, double* fp32_tflops, double* fp64_tflops);
cudaError_t launch_wait_probe(unsigned long long limit_ns, unsigned* errors, cudaStream_t s);

cudaError_t launch_read_fields(const void* fields, int precision, int n_pix, int n_bins, void* E,
                               void* B, int dtype, cudaStream_t s);
cudaError_t launch_write_fields(void* fields, int precision, int n_pix, int n_bins, const void* E, const void* B,
                                int dtype, cudaStream_t s);
// power spectra (rd_spectrum.cu): twiddles exp(-2 pi i j / N), j < N/2, computed on the host
void fill_twiddles(float2* host, int N);
constexpr int kFusedMaxN = 8192;   // longest series transformed in shared memory (24.5 N bytes per CTA)
bool spectrum_fused(int N);
cudaError_t launch_power_spectrum(const void* fields, int precision, int n_pix, int N, int c0, float2* z,
                                  float2* y, const float2* tw, float scale, float* P, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// device helpers: mbarrier, bulk async copy, vector reductions
// ---------------------------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy (TMA unit, non-tensor form); completes on the mbarrier.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for an mbarrier phase for at most limit_ns; false if it did not complete in time.
__device__ __forceinline__ bool mbar_wait_bounded_ns(uint64_t* bar, unsigned parity, unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity)
{
    return mbar_wait_bounded_ns(bar, parity, kWaitLimitNs);
}

// Fire-and-forget vector reductions into global memory (sm_90+).
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

// Predicated forms: no memory access at all when `on` is false (the address is then not used).
__device__ __forceinline__ void red_add_v4_if(bool on, float* addr, float a, float b, float c, float d)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %5, 0;\n\t"
        "@p red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(addr),
        "f"(a), "f"(b), "f"(c), "f"(d), "r"((unsigned)on)
        : "memory");
}

__device__ __forceinline__ void red_add_v2_if(bool on, float* addr, float a, float b)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\t"
        "@p red.global.add.v2.f32 [%0], {%1, %2};\n\t}" ::"l"(addr),
        "f"(a), "f"(b), "r"((unsigned)on)
        : "memory");
}

__device__ __forceinline__ void red_add_v2(float* addr, float a, float b)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}

__device__ __forceinline__ void red_add_f64(double* addr, double v)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(addr), "d"(v) : "memory");
}

// Single-instruction approximations (relative error about 1 ulp, denormals flushed).
__device__ __forceinline__ float fast_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float fast_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// =============================================================================================
// Eq. 2 in bin units, FP64, every operation separately rounded:
//   t_k = t0 + k*dt,  R = sqrt((dx*dx + dy*dy) + dz*dz),  u = ((t_k + R) - T0) * inv_dt_det
// =============================================================================================
__device__ __forceinline__ double arrival_bins(double xk0, double xk1, double xk2, const D4& cell,
                                               double t0, int k, double dt, double inv_dt_det,
                                               double& R)
{
    const double dx = __dsub_rn(cell.x, xk0);
    const double dy = __dsub_rn(cell.y, xk1);
    const double dz = __dsub_rn(cell.z, xk2);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    R = __dsqrt_rn(r2);
    const double tk = __dadd_rn(t0, __dmul_rn((double)k, dt));
    return __dmul_rn(__dsub_rn(__dadd_rn(tk, R), cell.w), inv_dt_det);
}

// Far-field limit: the cell seen from the origin along n_c = P/R_c at R_c = |P|, computed as
// R_c = sqrt((x*x + y*y) + z*z), n_c = P / R_c (separately rounded).
__device__ __forceinline__ void farfield_cell(const D4& cell, double& nx, double& ny, double& nz, double& Rc)
{
    Rc = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(cell.x, cell.x), __dmul_rn(cell.y, cell.y)),
                              __dmul_rn(cell.z, cell.z)));
    nx = __ddiv_rn(cell.x, Rc);
    ny = __ddiv_rn(cell.y, Rc);
    nz = __ddiv_rn(cell.z, Rc);
}

// Eq. 3 in bin units, FP64, every operation separately rounded:
//   u = (((t0 + k*dt) + R_c) - ((x*nx + y*ny) + z*nz) - T0) * inv_dt_det
__device__ __forceinline__ double arrival_bins_ff(double xk0, double xk1, double xk2, double nx, double ny,
                                                  double nz, double Rc, double T0, double t0, int k, double dt,
                                                  double inv_dt_det)
{
    const double tk = __dadd_rn(t0, __dmul_rn((double)k, dt));
    const double xn = __dadd_rn(__dadd_rn(__dmul_rn(xk0, nx), __dmul_rn(xk1, ny)), __dmul_rn(xk2, nz));
    return __dmul_rn(__dsub_rn(__dsub_rn(__dadd_rn(tk, Rc), xn), T0), inv_dt_det);
}

__device__ __forceinline__ int clamp_bin(double fb)
{
    return (int)fmin(fmax(fb, -1073741824.0), 1073741824.0);
}

#endif

}  // namespace rd
