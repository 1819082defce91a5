// Host side of the C ABI declared in include/rd.h: argument checks, device memory of the
// detector, per-call scratch, particle chunking and kernel launches.  No entry point allocates
// on the hot path once a detector's scratch has reached the working size.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "rd_internal.cuh"

using namespace rd;

static constexpr size_t kBatchBudgetDefault = (size_t)4 << 30;   // records per batch launch group

struct rd_detector {
    int device = 0;
    int n_pix = 0;
    int n_bins = 0;
    int precision = RD_MIXED;
    int flags = RD_NEAR | RD_FAR;
    double t_min = 0.0;
    double dt_det = 1.0;
    D4* cells = nullptr;             // [n_pix]
    void* fields = nullptr;          // internal accumulators
    size_t field_bytes = 0;
    DevCounters* counters = nullptr;
    DevCounters* host_counters = nullptr;   // page-locked copy target of `counters`
    void* rec = nullptr;             // per-sample records
    size_t rec_bytes = 0;
    void* stage = nullptr;           // device copy of host trajectories
    size_t stage_bytes = 0;
    void* readback = nullptr;        // conversion buffer for host reads
    size_t readback_bytes = 0;
    void* seed = nullptr;            // adjoint: upstream gradient in field layout
    size_t seed_bytes = 0;
    void* gbeta = nullptr;           // adjoint: d loss / d beta (FP64)
    size_t gbeta_bytes = 0;
    int adjoint_chunk = 250;         // adjoint: samples between recomputed anchors
    int adjoint_mode = RD_ADJ_FP32;  // RD_MIXED adjoint: FP32 or compensated (double-float) kernel
    unsigned long long id = 0;       // unique per created detector (keys of cached graphs)
    // batched form (kept in the first detector of a batch)
    void* batch_rec = nullptr;       // records of every problem
    size_t batch_rec_bytes = 0;
    void* batch_tab = nullptr;       // DepositParams per segment + item offsets + a counter per group
    size_t batch_tab_bytes = 0;
    size_t batch_budget = kBatchBudgetDefault;   // bytes of records per launch group
    void* spec = nullptr;            // power spectra: two complex work arrays
    size_t spec_bytes = 0;
    void* spec_tw = nullptr;         // twiddles of length spec_n
    size_t spec_tw_bytes = 0;
    int spec_n = 0;
    std::vector<float2> spec_tw_host;
    // streamed deposits: the last sample (x, u) of every particle from the previous call
    void* strm_last = nullptr;       // x then u, each [n_part][3][3] doubles (last samples)
    size_t strm_last_bytes = 0;
    void* strm_stage = nullptr;      // this call's samples with the stored one in front, and q
    size_t strm_stage_bytes = 0;
    int strm_n_part = -1;            // -1: no stream in progress
    int strm_have = 0;               // samples kept per particle (1; 2 with RD_LINEAR / RD_HOLD_PREV; 3 with
                                     // RD_QUADRATIC)
    long long strm_count = 0;        // samples of the stream handed over so far
    double strm_t_last = 0.0;
    double strm_dt = 0.0;
    std::vector<unsigned long long> graph_key;
    cudaGraphExec_t graph_exec = nullptr;
    long long n_deposits = 0;
    int chunk_override = 0;          // intervals per work item (0 = automatic)
    int group_override = 0;          // cell blocks per work-order group (0 = automatic)
    int cpc = kMixedCellsPerCta;     // RD_MIXED deposit shape: cells per CTA ...
    int nc = kMixedCells;            // ... and cells per thread
    bool timing = false;             // record CUDA events around deposit launches
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending, ev_free;
    long long timed_launches = 0;
    double timed_ms = 0.0;
};

namespace {

thread_local std::string g_err;
unsigned long long g_next_id = 1;   // detector ids (host side, monotonic)

rd_status fail(rd_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

rd_status cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(RD_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(RD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define RD_CUDA(call, what)                              \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Grow a scratch buffer (contents not kept).  Waits for the stream before freeing the old one.
rd_status ensure(void** buf, size_t* have, size_t need, cudaStream_t s, const char* what)
{
    if (*have >= need) return RD_OK;
    if (*buf) {
        RD_CUDA(cudaStreamSynchronize(s), what);
        RD_CUDA(cudaFree(*buf), what);
        *buf = nullptr;
        *have = 0;
    }
    size_t bytes = std::max(need, (size_t)(1u << 20));
    RD_CUDA(cudaMalloc(buf, bytes), what);
    *have = bytes;
    return RD_OK;
}

rd_status latched(const DevCounters& c)
{
    if (c.errors & ERRBIT_INPUT)
        return fail(RD_ERR_INPUT, "trajectory rejected: a chord speed |x_k - x_{k-1}|/dt >= 1 or a "
                                  "non-finite sample");
    if (c.errors & ERRBIT_TIMEOUT)
        return fail(RD_ERR_TIMEOUT, "a kernel's bounded wait ran out; its work was abandoned");
    if (c.errors & ERRBIT_BOUNDS) return fail(RD_ERR_BOUNDS, "a kernel index left the detector");
    return RD_OK;
}

rd_status check_traj(const rd_traj* t)
{
    if (!t) return fail(RD_ERR_ARG, "traj is NULL");
    if (t->n_part < 0 || t->n_samples < 1)
        return fail(RD_ERR_ARG, "bad trajectory shape n_part=%d n_samples=%d", t->n_part, t->n_samples);
    if (!(t->dt > 0.0) || !isfinite(t->dt) || !isfinite(t->t0))
        return fail(RD_ERR_ARG, "dt must be finite and > 0 and t0 finite");
    if (t->mem != RD_MEM_DEVICE && t->mem != RD_MEM_HOST) return fail(RD_ERR_ARG, "bad traj->mem");
    if (t->n_part > 0 && (!t->x || !t->u)) return fail(RD_ERR_ARG, "traj x/u is NULL");
    return RD_OK;
}

// Intervals per work item: the detector's override, else the default rule.
int choose_chunk(const rd_detector* d, int n_part, int S, int n_cell_blocks)
{
    if (d->chunk_override > 0) return std::min(d->chunk_override, S);
    return auto_chunk(n_cell_blocks, n_part, S);
}

// Bracket one deposit-kernel launch with events when timing is on.
struct LaunchTimer {
    rd_detector* d;
    cudaStream_t s;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    LaunchTimer(rd_detector* d_, cudaStream_t s_) : d(d_), s(s_)
    {
        if (!d->timing) return;
        if (!d->ev_free.empty()) {
            ev = d->ev_free.back();
            d->ev_free.pop_back();
        } else if (cudaEventCreate(&ev.first) != cudaSuccess || cudaEventCreate(&ev.second) != cudaSuccess) {
            ev = {nullptr, nullptr};
            return;
        }
        cudaEventRecord(ev.first, s);
    }
    ~LaunchTimer()
    {
        if (!ev.first) return;
        cudaEventRecord(ev.second, s);
        d->ev_pending.push_back(ev);
    }
};

void collect_timings(rd_detector* d)
{
    for (auto& ev : d->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) {
            d->timed_ms += ms;
            d->timed_launches += 1;
        }
        d->ev_free.push_back(ev);
    }
    d->ev_pending.clear();
}

void fill_mixed_params(DepositParams& P, const rd_detector* d, const rd_traj* t, const void* rec,
                       const double* x, const double* q, int np, int chunk)
{
    const int S = t->n_samples - 1;
    P.rec = rec;
    P.x = x;
    P.q = q;
    P.cells = d->cells;
    P.fields = d->fields;
    P.counters = d->counters;
    P.n_pix = d->n_pix;
    P.n_bins = d->n_bins;
    P.n_samples = t->n_samples;
    P.n_part = np;
    P.chunk = chunk;
    P.k_first = 1;
    P.n_chunks = (S + chunk - 1) / chunk;
    P.n_cell_blocks = (d->n_pix + kMixedCellsPerCta - 1) / kMixedCellsPerCta;
    P.t0 = t->t0;
    P.dt = t->dt;
    P.inv_dt_det = 1.0 / d->dt_det;
    P.dt_f = (float)t->dt;
    P.du_scale = (float)(t->dt / d->dt_det);
    P.ff = (d->flags & RD_FARFIELD) != 0;
    P.lin = (d->flags & RD_LINEAR) ? 1 : (d->flags & RD_HOLD_PREV) ? 2 : (d->flags & RD_QUADRATIC) ? 3 : 0;
    P.W = (float)(d->dt_det / t->dt);
    P.invW = (float)(t->dt / d->dt_det);
    P.cpc = kMixedCellsPerCta;
    P.nc = kMixedCells;
    P.group = d->group_override > 0 ? std::min(d->group_override, P.n_cell_blocks)
                                    : cell_group(P.n_cell_blocks, d->n_bins, kMixedCellsPerCta, chunk, S);
}

}  // namespace

namespace rd {
// Last-error message for entry points defined in other translation units.
rd_status set_last_error(rd_status st, const char* msg)
{
    g_err = msg ? msg : "";
    return st;
}

int sm_count()
{
    constexpr int kMaxDev = 256;
    static std::atomic<int> cache[kMaxDev];        // 0: not queried yet
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < kMaxDev && (n = cache[dev].load(std::memory_order_relaxed)) > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    if (dev >= 0 && dev < kMaxDev) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

int grid_stride_blocks(long long n, int threads, int per_sm)
{
    long long g = (n + threads - 1) / threads;
    g = std::min(g, (long long)sm_count() * per_sm);
    return (int)std::max(1LL, g);
}

int auto_chunk(long long n_cell_blocks, long long n_part, int S)
{
    int chunk = std::min(kDefaultChunk, S);
    const long long want = 8LL * sm_count();       // resident CTAs for a few waves
    while (chunk > 64 && n_cell_blocks * n_part * ((S + chunk - 1) / chunk) < want) chunk /= 2;
    return std::max(1, chunk);
}

int cell_group(int n_cell_blocks, int n_bins, int cells_per_cta, int chunk, int n_intervals)
{
#ifdef RD_GROUP
    return std::max(1, std::min(n_cell_blocks, RD_GROUP));
#else
#ifndef RD_GROUP_SLICE_MB
#define RD_GROUP_SLICE_MB 70
#endif
    // a chunk's arrivals span about its share of the trajectory's bins (the window holds every
    // arrival), and the resident CTAs, at different points of their chunks, a quarter more
    const double span = std::min(1.0, 1.25 * (double)chunk / (double)std::max(1, n_intervals));
    const double slice = (double)cells_per_cta * n_bins * 32.0 * span;
    const int g = (int)((double)RD_GROUP_SLICE_MB * 1048576.0 / slice);
    return std::max(1, std::min(std::min(n_cell_blocks, 8), g));
#endif
}

const char* flags_error(int flags)
{
    if (flags & ~(RD_NEAR | RD_FAR | RD_FARFIELD | RD_LINEAR | RD_HOLD_PREV | RD_QUADRATIC)) return "unknown flag bits";
    const int interp = flags & (RD_LINEAR | RD_HOLD_PREV | RD_QUADRATIC);
    if (interp & (interp - 1)) return "RD_LINEAR, RD_HOLD_PREV and RD_QUADRATIC are alternatives";
    if ((flags & (RD_NEAR | RD_FAR)) == 0 && flags != 0)
        return "flags select no term of Eq. 1 (RD_NEAR and/or RD_FAR)";
    if ((flags & RD_FARFIELD) && (flags & RD_NEAR))
        return "RD_FARFIELD keeps only the radiation term: RD_NEAR cannot be combined with it";
    return nullptr;
}
}  // namespace rd

extern "C" {

const char* rd_last_error(void) { return g_err.c_str(); }

const char* rd_version(void) { return "rd 0.1 (sm_103a)"; }

rd_status rd_push_boris(int32_t n_part, int32_t n_steps, double dt, const double* B, double qm, double* x,
                        double* u, double* x_out, double* u_out, rd_stream stream)
{
    g_err.clear();
    if (n_part < 0 || n_steps < 0) return fail(RD_ERR_ARG, "negative count (n_part %d, n_steps %d)", n_part, n_steps);
    if (!B || !isfinite(dt) || !isfinite(qm) || !isfinite(B[0]) || !isfinite(B[1]) || !isfinite(B[2]))
        return fail(RD_ERR_ARG, "B is NULL, or dt, qm or B not finite");
    if (n_part == 0 || n_steps == 0) return RD_OK;
    if (!x || !u || !x_out || !u_out) return fail(RD_ERR_ARG, "state or output pointer is NULL");
    RD_CUDA(launch_push_boris(n_part, n_steps, dt, B, qm, x, u, x_out, u_out, reinterpret_cast<cudaStream_t>(stream)),
            "rd_push_boris");
    return RD_OK;
}

rd_status rd_check_bounded_wait(int32_t limit_ms, rd_stream stream)
{
    g_err.clear();
    if (limit_ms < 1 || limit_ms > 2000) return fail(RD_ERR_ARG, "limit_ms %d outside [1, 2000]", limit_ms);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned* dev = nullptr;
    RD_CUDA(cudaMalloc(&dev, sizeof(unsigned)), "rd_check_bounded_wait");
    DevCounters c{};
    cudaError_t e = cudaMemsetAsync(dev, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = launch_wait_probe((unsigned long long)limit_ms * 1000000ull, dev, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c.errors, dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dev);
    RD_CUDA(e, "rd_check_bounded_wait");
    const rd_status st = latched(c);
    if (st == RD_OK) return fail(RD_ERR_STATE, "the bounded wait did not report its expiry");
    return st;
}

rd_status rd_measure_fma_peaks(double* fp32_tflops, double* fp64_tflops, rd_stream stream)
{
    g_err.clear();
    if (fp32_tflops) *fp32_tflops = 0.0;
    if (fp64_tflops) *fp64_tflops = 0.0;
    RD_CUDA(measure_fma_peaks(reinterpret_cast<cudaStream_t>(stream), fp32_tflops, fp64_tflops),
            "rd_measure_fma_peaks");
    return RD_OK;
}

rd_status rd_create_detector(const rd_detector_desc* desc, rd_stream stream, rd_detector** out)
{
    g_err.clear();
    if (!desc || !out) return fail(RD_ERR_ARG, "desc/out is NULL");
    *out = nullptr;
    if (desc->n_pix < 1 || desc->n_bins < 1)
        return fail(RD_ERR_ARG, "n_pix and n_bins must be >= 1 (got %d, %d)", desc->n_pix, desc->n_bins);
    if (!desc->pix_pos) return fail(RD_ERR_ARG, "pix_pos is NULL");
    if (!(desc->dt_det > 0.0) || !isfinite(desc->dt_det) || !isfinite(desc->t_min))
        return fail(RD_ERR_ARG, "dt_det must be finite and > 0, t_min finite");
    if (desc->precision != RD_MIXED && desc->precision != RD_FP64)
        return fail(RD_ERR_ARG, "bad precision %d", desc->precision);
    if (desc->mem != RD_MEM_DEVICE && desc->mem != RD_MEM_HOST) return fail(RD_ERR_ARG, "bad desc->mem");
    if (const char* why = flags_error(desc->flags)) return fail(RD_ERR_ARG, "bad flags %d: %s", desc->flags, why);
    if (desc->precision == RD_MIXED && desc->n_bins > kMixedMaxBins)
        return fail(RD_ERR_ARG, "an RD_MIXED detector holds at most %d bins per cell (got %d)", kMixedMaxBins,
                    desc->n_bins);
    const size_t per_bin = desc->precision == RD_MIXED ? 8 * sizeof(float) : 6 * sizeof(double);
    if ((size_t)desc->n_pix * (size_t)desc->n_bins > ((size_t)1 << 40) / per_bin)
        return fail(RD_ERR_ARG, "detector too large");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    // cell table on the host: (x, y, z, T0 = t_min + pix_t0)
    std::vector<double> pos((size_t)desc->n_pix * 3), t0v;
    if (desc->mem == RD_MEM_HOST) {
        memcpy(pos.data(), desc->pix_pos, pos.size() * sizeof(double));
    } else {
        RD_CUDA(cudaMemcpy(pos.data(), desc->pix_pos, pos.size() * sizeof(double), cudaMemcpyDeviceToHost),
                "copy pix_pos");
    }
    if (desc->pix_t0) {
        t0v.resize(desc->n_pix);
        if (desc->mem == RD_MEM_HOST)
            memcpy(t0v.data(), desc->pix_t0, t0v.size() * sizeof(double));
        else
            RD_CUDA(cudaMemcpy(t0v.data(), desc->pix_t0, t0v.size() * sizeof(double), cudaMemcpyDeviceToHost),
                    "copy pix_t0");
    }
    std::vector<D4> cells(desc->n_pix);
    for (int j = 0; j < desc->n_pix; ++j) {
        const double T0 = desc->t_min + (desc->pix_t0 ? t0v[j] : 0.0);
        cells[j] = D4{pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], T0};
        if (!isfinite(cells[j].x) || !isfinite(cells[j].y) || !isfinite(cells[j].z) || !isfinite(T0))
            return fail(RD_ERR_ARG, "cell %d has a non-finite position or time origin", j);
    }

    rd_detector* d = new (std::nothrow) rd_detector();
    if (!d) return fail(RD_ERR_OOM, "host allocation");
    cudaGetDevice(&d->device);
    d->id = __atomic_fetch_add(&g_next_id, 1ull, __ATOMIC_RELAXED);
    d->n_pix = desc->n_pix;
    d->n_bins = desc->n_bins;
    d->precision = desc->precision;
    d->flags = desc->flags ? desc->flags : (RD_NEAR | RD_FAR);
    d->t_min = desc->t_min;
    d->dt_det = desc->dt_det;
    d->field_bytes = (size_t)desc->n_pix * desc->n_bins * per_bin;
    cudaError_t e = cudaMalloc(&d->cells, sizeof(D4) * cells.size());
    if (e == cudaSuccess) e = cudaMalloc(&d->fields, d->field_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d->counters, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMallocHost(&d->host_counters, sizeof(DevCounters));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d->cells, cells.data(), sizeof(D4) * cells.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->fields, 0, d->field_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->counters, 0, sizeof(DevCounters), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        rd_status st = cuda_fail(e, "rd_create_detector");
        cudaFree(d->cells);
        cudaFree(d->fields);
        cudaFree(d->counters);
        cudaFreeHost(d->host_counters);
        delete d;
        return st;
    }
    *out = d;
    return RD_OK;
}

rd_status rd_destroy(rd_detector* d)
{
    g_err.clear();
    if (!d) return RD_OK;
    cudaDeviceSynchronize();
    for (auto& ev : d->ev_pending) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
    for (auto& ev : d->ev_free) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
    cudaFree(d->cells);
    cudaFree(d->fields);
    cudaFree(d->counters);
    cudaFreeHost(d->host_counters);
    cudaFree(d->rec);
    cudaFree(d->stage);
    cudaFree(d->readback);
    cudaFree(d->seed);
    cudaFree(d->gbeta);
    cudaFree(d->batch_rec);
    cudaFree(d->batch_tab);
    cudaFree(d->strm_last);
    cudaFree(d->strm_stage);
    cudaFree(d->spec);
    cudaFree(d->spec_tw);
    if (d->graph_exec) cudaGraphExecDestroy(d->graph_exec);
    delete d;
    return RD_OK;
}

rd_status rd_zero_fields(rd_detector* d, rd_stream stream)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    RD_CUDA(cudaMemsetAsync(d->fields, 0, d->field_bytes, s), "rd_zero_fields");
    RD_CUDA(cudaMemsetAsync(&d->counters->clipped, 0, 2 * sizeof(unsigned long long), s), "rd_zero_fields");
    d->n_deposits = 0;
    return RD_OK;
}

// Deposit intervals k_first..S of t (k_first > 1: the earlier samples only provide the
// previous quantities, used by streamed calls).
static rd_status deposit_from(rd_detector* d, const rd_traj* t, rd_stream stream, int k_first, int k_real0 = 0)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    rd_status st = check_traj(t);
    if (st != RD_OK) return st;
    const int S = t->n_samples - 1;
    if (t->n_part == 0 || S < k_first) return RD_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool mixed = d->precision == RD_MIXED;
    const size_t rec_size = mixed ? sizeof(RecS) : sizeof(RecD);
    const size_t per_part_rec = rec_size * (size_t)t->n_samples;
    const size_t per_part_in = 2 * 3 * sizeof(double) * (size_t)t->n_samples + sizeof(double);
    // particle chunk: bounded scratch (records + staged input)
    const size_t budget = (size_t)1 << 31;
    const size_t per_part = per_part_rec + (t->mem == RD_MEM_HOST ? per_part_in : 0);
    int pc = (int)std::max<size_t>(1, std::min<size_t>((size_t)t->n_part, budget / per_part));
    st = ensure(&d->rec, &d->rec_bytes, per_part_rec * pc, s, "record scratch");
    if (st != RD_OK) return st;
    if (t->mem == RD_MEM_HOST) {
        st = ensure(&d->stage, &d->stage_bytes, per_part_in * pc + 256, s, "staging scratch");
        if (st != RD_OK) return st;
    }
    // RD_MIXED: the detector's shape (the far-field and interpolation variants run the default one)
    const bool def_shape = !mixed || (d->flags & (RD_FARFIELD | RD_LINEAR | RD_HOLD_PREV | RD_QUADRATIC));
    const int cpc = def_shape ? kMixedCellsPerCta : d->cpc, nc = def_shape ? kMixedCells : d->nc;
    static_assert(kDepositThreads == kMixedCellsPerCta, "both deposit kernels cover 256 cells per CTA");
    const int n_cell_blocks = (d->n_pix + (mixed ? cpc : kDepositThreads) - 1) / (mixed ? cpc : kDepositThreads);
    const int chunk = choose_chunk(d, std::min(pc, t->n_part), S - k_first + 1, n_cell_blocks);

    for (int p0 = 0; p0 < t->n_part; p0 += pc) {
        const int np = std::min(pc, t->n_part - p0);
        const size_t n3 = (size_t)np * t->n_samples * 3;
        const double* x = t->x + (size_t)p0 * t->n_samples * 3;
        const double* u = t->u + (size_t)p0 * t->n_samples * 3;
        const double* q = t->q ? t->q + p0 : nullptr;
        if (t->mem == RD_MEM_HOST) {
            double* sx = static_cast<double*>(d->stage);
            double* su = sx + n3;
            double* sq = su + n3;
            RD_CUDA(cudaMemcpyAsync(sx, x, n3 * sizeof(double), cudaMemcpyHostToDevice, s), "stage x");
            RD_CUDA(cudaMemcpyAsync(su, u, n3 * sizeof(double), cudaMemcpyHostToDevice, s), "stage u");
            if (q) RD_CUDA(cudaMemcpyAsync(sq, q, np * sizeof(double), cudaMemcpyHostToDevice, s), "stage q");
            x = sx;
            u = su;
            q = q ? sq : nullptr;
        }
        DepositParams P;
        P.rec = d->rec;
        P.x = x;
        P.q = q;
        P.cells = d->cells;
        P.fields = d->fields;
        P.counters = d->counters;
        P.n_pix = d->n_pix;
        P.n_bins = d->n_bins;
        P.n_samples = t->n_samples;
        P.n_part = np;
        P.chunk = chunk;
        P.k_first = k_first;
        P.k_real0 = k_real0;
        P.n_chunks = (S - k_first + chunk) / chunk;
        P.n_cell_blocks = n_cell_blocks;
        P.t0 = t->t0;
        P.dt = t->dt;
        P.inv_dt_det = 1.0 / d->dt_det;
        P.dt_f = (float)t->dt;
        P.du_scale = (float)(t->dt / d->dt_det);
        P.W = (float)(d->dt_det / t->dt);
        P.invW = (float)(t->dt / d->dt_det);
        P.ff = (d->flags & RD_FARFIELD) != 0;
        P.lin = (d->flags & RD_LINEAR) ? 1 : (d->flags & RD_HOLD_PREV) ? 2 : (d->flags & RD_QUADRATIC) ? 3 : 0;
        P.cpc = cpc;
        P.nc = nc;
        P.group = !mixed ? 1
                         : d->group_override > 0 ? std::min(d->group_override, n_cell_blocks)
                                                 : cell_group(n_cell_blocks, d->n_bins, cpc, chunk, S - k_first + 1);
        if (mixed) {
            RD_CUDA(launch_precompute_mixed(x, u, q, t->dt / d->dt_det, np, t->n_samples, t->dt, d->flags,
                                            static_cast<RecS*>(d->rec), d->counters, s),
                    "precompute");
            LaunchTimer timer(d, s);
            RD_CUDA(launch_deposit_mixed(P, s), "deposit (mixed)");
        } else {
            RD_CUDA(launch_precompute_fp64(x, u, q, np, t->n_samples, t->t0, t->dt, d->flags,
                                           static_cast<RecD*>(d->rec), d->counters, s),
                    "precompute");
            LaunchTimer timer(d, s);
            RD_CUDA(launch_deposit_fp64(P, d->flags, s), "deposit (fp64)");
        }
    }
    d->n_deposits += (long long)t->n_part * (S - k_first + 1) * d->n_pix;
    return RD_OK;
}

rd_status rd_deposit_trajectories(rd_detector* d, const rd_traj* t, rd_stream stream)
{
    return deposit_from(d, t, stream, 1);
}

rd_status rd_read_fields(rd_detector* d, void* E, void* B, int32_t dtype, int32_t mem, rd_stream stream)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    if (dtype != RD_F32 && dtype != RD_F64) return fail(RD_ERR_ARG, "bad dtype %d", dtype);
    if (mem != RD_MEM_DEVICE && mem != RD_MEM_HOST && mem != RD_MEM_HOST_ASYNC) return fail(RD_ERR_ARG, "bad mem %d", mem);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!E && !B) return RD_OK;
    const size_t elem = dtype == RD_F32 ? sizeof(float) : sizeof(double);
    const size_t one = (size_t)d->n_pix * d->n_bins * 3 * elem;
    if (mem == RD_MEM_DEVICE) {
        RD_CUDA(launch_read_fields(d->fields, d->precision, d->n_pix, d->n_bins, E, B, dtype, s),
                "rd_read_fields");
        return RD_OK;
    }
    rd_status st = ensure(&d->readback, &d->readback_bytes, 2 * one, s, "readback scratch");
    if (st != RD_OK) return st;
    char* dE = E ? static_cast<char*>(d->readback) : nullptr;
    char* dB = B ? static_cast<char*>(d->readback) + one : nullptr;
    RD_CUDA(launch_read_fields(d->fields, d->precision, d->n_pix, d->n_bins, dE, dB, dtype, s),
            "rd_read_fields");
    if (E) RD_CUDA(cudaMemcpyAsync(E, dE, one, cudaMemcpyDeviceToHost, s), "copy E to host");
    if (B) RD_CUDA(cudaMemcpyAsync(B, dB, one, cudaMemcpyDeviceToHost, s), "copy B to host");
    if (mem == RD_MEM_HOST_ASYNC) return RD_OK;
    RD_CUDA(cudaMemcpyAsync(d->host_counters, d->counters, sizeof(DevCounters), cudaMemcpyDeviceToHost, s),
            "read counters");
    RD_CUDA(cudaStreamSynchronize(s), "rd_read_fields");
    return latched(*d->host_counters);
}

rd_status rd_write_fields(rd_detector* d, const void* E, const void* B, int32_t dtype, int32_t mem, rd_stream stream)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    if (dtype != RD_F32 && dtype != RD_F64) return fail(RD_ERR_ARG, "bad dtype %d", dtype);
    if (mem != RD_MEM_DEVICE && mem != RD_MEM_HOST && mem != RD_MEM_HOST_ASYNC) return fail(RD_ERR_ARG, "bad mem %d", mem);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (mem == RD_MEM_DEVICE) {
        RD_CUDA(launch_write_fields(d->fields, d->precision, d->n_pix, d->n_bins, E, B, dtype, s), "rd_write_fields");
        return RD_OK;
    }
    const size_t elem = dtype == RD_F32 ? sizeof(float) : sizeof(double);
    const size_t one = (size_t)d->n_pix * d->n_bins * 3 * elem;
    rd_status st = ensure(&d->readback, &d->readback_bytes, 2 * one, s, "field staging");
    if (st != RD_OK) return st;
    char* dE = E ? static_cast<char*>(d->readback) : nullptr;
    char* dB = B ? static_cast<char*>(d->readback) + one : nullptr;
    if (E) RD_CUDA(cudaMemcpyAsync(dE, E, one, cudaMemcpyHostToDevice, s), "copy E to the device");
    if (B) RD_CUDA(cudaMemcpyAsync(dB, B, one, cudaMemcpyHostToDevice, s), "copy B to the device");
    RD_CUDA(launch_write_fields(d->fields, d->precision, d->n_pix, d->n_bins, dE, dB, dtype, s), "rd_write_fields");
    if (mem == RD_MEM_HOST) RD_CUDA(cudaStreamSynchronize(s), "rd_write_fields");
    return RD_OK;
}

rd_status rd_synchronize(rd_detector* d, rd_stream stream)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    RD_CUDA(cudaMemcpyAsync(d->host_counters, d->counters, sizeof(DevCounters), cudaMemcpyDeviceToHost, s),
            "read counters");
    RD_CUDA(cudaStreamSynchronize(s), "rd_synchronize");
    const DevCounters c = *d->host_counters;
    if (c.errors) {
        RD_CUDA(cudaMemsetAsync(&d->counters->errors, 0, sizeof(unsigned), s), "clear errors");
        RD_CUDA(cudaStreamSynchronize(s), "rd_synchronize");
    }
    return latched(c);
}

rd_status rd_get_stats(rd_detector* d, rd_stream stream, rd_stats* out)
{
    g_err.clear();
    if (!d || !out) return fail(RD_ERR_ARG, "detector/out is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    RD_CUDA(cudaMemcpyAsync(d->host_counters, d->counters, sizeof(DevCounters), cudaMemcpyDeviceToHost, s),
            "read counters");
    RD_CUDA(cudaStreamSynchronize(s), "rd_get_stats");
    const DevCounters c = *d->host_counters;
    out->n_clipped = (int64_t)c.clipped;
    out->n_bin_crossings = (int64_t)c.crossings;
    out->n_deposits = d->n_deposits;
    out->device_errors = c.errors;
    collect_timings(d);
    out->kernel_launches = d->timed_launches;
    out->kernel_ms = d->timed_ms;
    d->timed_launches = 0;
    d->timed_ms = 0.0;
    return RD_OK;
}

// Compensated adjoint of an RD_MIXED detector (rd_adjoint_comp.cu): double-float records, the
// kernel adds d L / d x and d L / d u to gx and gu directly.
static rd_status adjoint_compensated(rd_detector* d, const rd_traj* t, const void* gE, const void* gB,
                                     int32_t gdtype, double* gx, double* gu, cudaStream_t s)
{
    const int S = t->n_samples - 1;
    rd_status st = ensure(&d->seed, &d->seed_bytes, 2 * d->field_bytes, s, "seed scratch");   // 64 B per bin
    if (st != RD_OK) return st;
    RD_CUDA(launch_pack_seed_df(gE, gB, gdtype, d->n_pix, d->n_bins, static_cast<float*>(d->seed), s), "pack seed");
    const size_t per_part_rec = comp_record_bytes() * (size_t)t->n_samples;
    const size_t budget = (size_t)1 << 31;
    const int pc = (int)std::max<size_t>(1, std::min<size_t>((size_t)t->n_part, budget / per_part_rec));
    st = ensure(&d->rec, &d->rec_bytes, per_part_rec * pc, s, "record scratch");
    if (st != RD_OK) return st;
    const int n_cell_blocks = (d->n_pix + kAdjointCompThreads - 1) / kAdjointCompThreads;
    const int chunk = std::max(1, std::min(d->adjoint_chunk, S));
    for (int p0 = 0; p0 < t->n_part; p0 += pc) {
        const int np = std::min(pc, t->n_part - p0);
        const size_t off = (size_t)p0 * t->n_samples * 3;
        RD_CUDA(launch_precompute_comp(t->x + off, t->u + off, np, t->n_samples, t->dt, d->flags, d->rec, d->counters,
                                       s),
                "precompute");
        AdjointParams P{};
        P.recc = d->rec;
        P.x = t->x + off;
        P.q = t->q ? t->q + p0 : nullptr;
        P.cells = d->cells;
        P.seed = static_cast<const float*>(d->seed);
        P.gx = gx + off;
        P.gu = gu + off;
        P.counters = d->counters;
        P.n_pix = d->n_pix;
        P.n_bins = d->n_bins;
        P.n_samples = t->n_samples;
        P.n_part = np;
        P.chunk = chunk;
        P.n_chunks = (S + chunk - 1) / chunk;
        P.n_cell_blocks = n_cell_blocks;
        P.flags = d->flags;
        P.t0 = t->t0;
        P.dt = t->dt;
        P.inv_dt_det = 1.0 / d->dt_det;
        LaunchTimer timer(d, s);
        RD_CUDA(launch_adjoint_comp(P, s), "adjoint (compensated)");
    }
    return RD_OK;
}

rd_status rd_adjoint_trajectories(rd_detector* d, const rd_traj* t, const void* gE, const void* gB,
                                  int32_t gdtype, double* gx, double* gu, rd_stream stream)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    rd_status st = check_traj(t);
    if (st != RD_OK) return st;
    if (d->flags & (RD_FARFIELD | RD_LINEAR | RD_HOLD_PREV | RD_QUADRATIC))
        return fail(RD_ERR_STATE, "the adjoint covers the exact fields with the held interpolation only");
    if (t->mem != RD_MEM_DEVICE) return fail(RD_ERR_ARG, "the adjoint needs device trajectories");
    if (!gE && !gB) return fail(RD_ERR_ARG, "gE and gB are both NULL");
    if (gdtype != RD_F32 && gdtype != RD_F64) return fail(RD_ERR_ARG, "bad gdtype %d", gdtype);
    if (t->n_part > 0 && (!gx || !gu)) return fail(RD_ERR_ARG, "gx/gu is NULL");
    const int S = t->n_samples - 1;
    if (t->n_part == 0 || S < 1) return RD_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool fp64 = d->precision == RD_FP64;
    if (!fp64 && d->adjoint_mode == RD_ADJ_COMPENSATED) return adjoint_compensated(d, t, gE, gB, gdtype, gx, gu, s);
    st = ensure(&d->seed, &d->seed_bytes, d->field_bytes, s, "seed scratch");
    if (st != RD_OK) return st;
    if (fp64)
        RD_CUDA(launch_pack_seed64(gE, gB, gdtype, d->n_pix, d->n_bins, static_cast<double*>(d->seed), s), "pack seed");
    else
        RD_CUDA(launch_pack_seed(gE, gB, gdtype, d->n_pix, d->n_bins, static_cast<float*>(d->seed), s), "pack seed");
    const size_t per_part_rec = (fp64 ? sizeof(RecD) : sizeof(RecS)) * (size_t)t->n_samples;
    const size_t per_part_gb = 3 * sizeof(double) * (size_t)t->n_samples;
    const size_t budget = (size_t)1 << 31;
    const int pc = (int)std::max<size_t>(1, std::min<size_t>((size_t)t->n_part, budget / (per_part_rec + per_part_gb)));
    st = ensure(&d->rec, &d->rec_bytes, per_part_rec * pc, s, "record scratch");
    if (st != RD_OK) return st;
    st = ensure(&d->gbeta, &d->gbeta_bytes, per_part_gb * pc, s, "gradient scratch");
    if (st != RD_OK) return st;
    const int cells_per_cta = fp64 ? kAdjointFp64Threads : kAdjointCellsPerCta;
    const int n_cell_blocks = (d->n_pix + cells_per_cta - 1) / cells_per_cta;
    const int chunk = std::max(1, std::min(d->adjoint_chunk, S));
    for (int p0 = 0; p0 < t->n_part; p0 += pc) {
        const int np = std::min(pc, t->n_part - p0);
        const size_t off = (size_t)p0 * t->n_samples * 3;
        RD_CUDA(cudaMemsetAsync(d->gbeta, 0, per_part_gb * np, s), "clear gradient scratch");
        if (fp64)
            RD_CUDA(launch_precompute_fp64(t->x + off, t->u + off, nullptr, np, t->n_samples, t->t0, t->dt,
                                           RD_NEAR | RD_FAR, static_cast<RecD*>(d->rec), d->counters, s),
                    "precompute");
        else
            RD_CUDA(launch_precompute_mixed(t->x + off, t->u + off, nullptr, 0.0, np, t->n_samples, t->dt, d->flags,
                                            static_cast<RecS*>(d->rec), d->counters, s),
                    "precompute");
        AdjointParams P;
        P.rec = fp64 ? nullptr : static_cast<const RecS*>(d->rec);
        P.recd = fp64 ? static_cast<const RecD*>(d->rec) : nullptr;
        P.seedd = fp64 ? static_cast<const double*>(d->seed) : nullptr;
        P.x = t->x + off;
        P.q = t->q ? t->q + p0 : nullptr;
        P.cells = d->cells;
        P.seed = fp64 ? nullptr : static_cast<const float*>(d->seed);
        P.gx = gx + off;
        P.gbeta = static_cast<double*>(d->gbeta);
        P.counters = d->counters;
        P.n_pix = d->n_pix;
        P.n_bins = d->n_bins;
        P.n_samples = t->n_samples;
        P.n_part = np;
        P.chunk = chunk;
        P.n_chunks = (S + chunk - 1) / chunk;
        P.n_cell_blocks = n_cell_blocks;
        P.flags = d->flags;
        P.t0 = t->t0;
        P.dt = t->dt;
        P.inv_dt_det = 1.0 / d->dt_det;
        P.dt_f = (float)t->dt;
        P.du_scale = (float)(t->dt / d->dt_det);
        P.W = (float)(d->dt_det / t->dt);
        P.invW = (float)(t->dt / d->dt_det);
        P.inv_dt_det_f = (float)(1.0 / d->dt_det);
        P.inv_dt_f = (float)(1.0 / t->dt);
        P.edge_tol = (float)(1e-4 * d->dt_det / t->dt);     // 1e-4 bin, ten times the walk's drift
        {
            LaunchTimer timer(d, s);
            RD_CUDA(fp64 ? launch_adjoint_fp64(P, s) : launch_adjoint_mixed(P, s), "adjoint");
        }
        RD_CUDA(launch_gbeta_to_gu(t->u + off, static_cast<const double*>(d->gbeta), gu + off,
                                   (long long)np * t->n_samples, s),
                "gradient to momenta");
    }
    return RD_OK;
}

rd_status rd_set_adjoint_mode(rd_detector* d, int32_t mode)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    if (mode != RD_ADJ_FP32 && mode != RD_ADJ_COMPENSATED) return fail(RD_ERR_ARG, "bad adjoint mode %d", mode);
    if (mode == RD_ADJ_COMPENSATED && d->precision != RD_MIXED)
        return fail(RD_ERR_STATE, "RD_ADJ_COMPENSATED applies to RD_MIXED detectors");
    d->adjoint_mode = mode;
    return RD_OK;
}

static rd_status shape_error(const rd_shape* sh)
{
    if (!sh) return fail(RD_ERR_ARG, "shape is NULL");
    if (!mixed_shape_supported(sh->cells_per_cta, sh->cells_per_thread))
        return fail(RD_ERR_ARG, "unsupported shape: %d cells per CTA, %d per thread (64/128/256 and 1/2)",
                    sh->cells_per_cta, sh->cells_per_thread);
    if (sh->chunk < 0 || sh->group < 0) return fail(RD_ERR_ARG, "chunk and group must be >= 0");
    return RD_OK;
}

rd_status rd_set_shape(rd_detector* d, const rd_shape* sh)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    rd_status st = shape_error(sh);
    if (st != RD_OK) return st;
    if (d->precision != RD_MIXED) return fail(RD_ERR_STATE, "shapes apply to RD_MIXED detectors");
    d->cpc = sh->cells_per_cta;
    d->nc = sh->cells_per_thread;
    d->chunk_override = sh->chunk;
    d->group_override = sh->group;
    return RD_OK;
}

rd_status rd_get_shape(const rd_detector* d, rd_shape* sh)
{
    g_err.clear();
    if (!d || !sh) return fail(RD_ERR_ARG, "detector/shape is NULL");
    sh->cells_per_cta = d->cpc;
    sh->cells_per_thread = d->nc;
    sh->chunk = d->chunk_override;
    sh->group = d->group_override;
    return RD_OK;
}

// Tuning-cache key: the device (name, multiprocessor count) and the problem.
static std::string shape_key(const rd_detector* d, const rd_traj* t)
{
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, d->device) != cudaSuccess) prop.name[0] = 0;
    char buf[512];
    snprintf(buf, sizeof buf, "%s|sm%d|pix%d|bins%d|part%d|int%d|flags%d", prop.name, prop.multiProcessorCount, d->n_pix,
             d->n_bins, t->n_part, t->n_samples - 1, d->flags);
    return buf;
}

rd_status rd_autotune_shape(rd_detector* d, const rd_traj* t, const char* cache_path, rd_stream stream,
                            rd_shape* chosen, int32_t* from_cache, double* ms_out)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    rd_status st = check_traj(t);
    if (st != RD_OK) return st;
    if (d->precision != RD_MIXED) return fail(RD_ERR_STATE, "shape tuning applies to RD_MIXED detectors");
    if (from_cache) *from_cache = 0;
    if (ms_out) *ms_out = 0.0;
    const int S = t->n_samples - 1;
    const std::string key = shape_key(d, t);
    if (cache_path) {
        std::map<std::string, TuneEntry> cache;
        std::string err;
        if (!tune_cache_load(cache_path, cache, err)) return fail(RD_ERR_ARG, "%s", err.c_str());
        const auto it = cache.find(key);
        if (it != cache.end()) {
            const rd_shape sh{it->second.cpc, it->second.nc, it->second.chunk, it->second.group};
            if (shape_error(&sh) != RD_OK) return fail(RD_ERR_ARG, "tuning cache entry %s is invalid", key.c_str());
            st = rd_set_shape(d, &sh);
            if (st != RD_OK) return st;
            if (from_cache) *from_cache = 1;
            if (ms_out) *ms_out = it->second.ms;
            if (chosen) *chosen = sh;
            return RD_OK;
        }
    }
    if (t->n_part == 0 || S < 1) return chosen ? rd_get_shape(d, chosen) : RD_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    RD_CUDA(cudaEventCreate(&e0), "autotune");
    RD_CUDA(cudaEventCreate(&e1), "autotune");
    rd_shape saved;
    rd_get_shape(d, &saved);
    const bool timing = d->timing;
    d->timing = false;
    rd_shape best = saved;
    float best_ms = -1.f;
    auto trial = [&](const rd_shape& sh) -> rd_status {
        rd_status r = rd_set_shape(d, &sh);
        if (r == RD_OK) r = rd_deposit_trajectories(d, t, stream);   // warm-up (also sizes the scratch)
        if (r == RD_OK) {
            cudaEventRecord(e0, s);
            r = rd_deposit_trajectories(d, t, stream);
            cudaEventRecord(e1, s);
        }
        if (r != RD_OK) return r;
        if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "autotune");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best = sh;
        }
        return RD_OK;
    };
    const bool variant = (d->flags & (RD_FARFIELD | RD_LINEAR | RD_HOLD_PREV | RD_QUADRATIC)) != 0;
    // 1. cells per CTA x cells per thread, automatic chunk and group
    for (int cpc : {256, 128, 64})
        for (int nc : {2, 1}) {
            if (variant && (cpc != kMixedCellsPerCta || nc != kMixedCells)) continue;
            if (st == RD_OK) st = trial(rd_shape{cpc, nc, 0, 0});
        }
    // 2. step chunk at the best shape
    const rd_shape b1 = best;
    for (int c : {512, 1024, 2048, 4096})
        if (st == RD_OK && c <= std::max(S, 512)) st = trial(rd_shape{b1.cells_per_cta, b1.cells_per_thread, std::min(c, S), 0});
    // 3. work-order group at the best shape and chunk
    const rd_shape b2 = best;
    const int n_cb = (d->n_pix + b2.cells_per_cta - 1) / b2.cells_per_cta;
    for (int g : {1, 2, 4, 8})
        if (st == RD_OK && g <= n_cb) st = trial(rd_shape{b2.cells_per_cta, b2.cells_per_thread, b2.chunk, g});
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    d->timing = timing;
    const rd_shape keep = st == RD_OK ? best : saved;
    rd_set_shape(d, &keep);
    const rd_status z = rd_zero_fields(d, stream);
    if (st != RD_OK) return st;
    if (cache_path) {
        std::string err;
        const TuneEntry e{best.cells_per_cta, best.cells_per_thread, best.chunk, best.group, (double)best_ms};
        if (!tune_cache_store(cache_path, key, e, err)) return fail(RD_ERR_ARG, "%s", err.c_str());
    }
    if (chosen) *chosen = best;
    if (ms_out) *ms_out = best_ms;
    return z;
}

rd_status rd_set_chunk(rd_detector* d, int32_t chunk)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    if (chunk < 0) return fail(RD_ERR_ARG, "chunk must be >= 0");
    d->chunk_override = chunk;
    return RD_OK;
}

rd_status rd_autotune(rd_detector* d, const rd_traj* t, rd_stream stream, int32_t* chosen)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    rd_status st = check_traj(t);
    if (st != RD_OK) return st;
    if (d->precision != RD_MIXED) return fail(RD_ERR_STATE, "autotuning applies to RD_MIXED detectors");
    const int S = t->n_samples - 1;
    if (t->n_part == 0 || S < 1) {
        if (chosen) *chosen = d->chunk_override;
        return RD_OK;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    RD_CUDA(cudaEventCreate(&e0), "autotune");
    RD_CUDA(cudaEventCreate(&e1), "autotune");
    const int saved = d->chunk_override;
    const bool timing = d->timing;
    d->timing = false;
    int best = 0;
    float best_ms = 0.f;
    for (int c = 64; c <= 4096; c *= 2) {
        const int chunk = std::min(c, S);
        d->chunk_override = chunk;
        st = rd_deposit_trajectories(d, t, stream);            // warm-up (also sizes the scratch)
        if (st == RD_OK) {
            cudaEventRecord(e0, s);
            st = rd_deposit_trajectories(d, t, stream);
            cudaEventRecord(e1, s);
        }
        if (st != RD_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = cuda_fail(cudaGetLastError(), "autotune"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best == 0 || ms < best_ms) {
            best = chunk;
            best_ms = ms;
        }
        if (chunk == S) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    d->timing = timing;
    d->chunk_override = (st == RD_OK) ? best : saved;
    const rd_status z = rd_zero_fields(d, stream);
    if (st != RD_OK) return st;
    if (chosen) *chosen = best;
    return z;
}

rd_status rd_deposit_batch(int32_t n, rd_detector* const* dets, const rd_traj* trajs, rd_stream stream)
{
    g_err.clear();
    if (n < 1 || !dets || !trajs) return fail(RD_ERR_ARG, "need n >= 1 detectors and trajectories");
    for (int i = 0; i < n; ++i) {
        if (!dets[i]) return fail(RD_ERR_ARG, "detector %d is NULL", i);
        if (dets[i]->precision != RD_MIXED) return fail(RD_ERR_STATE, "detector %d is not RD_MIXED", i);
        rd_status st = check_traj(&trajs[i]);
        if (st != RD_OK) return st;
        if (trajs[i].mem != RD_MEM_DEVICE) return fail(RD_ERR_ARG, "batch trajectories must be in device memory");
        if (dets[i]->device != dets[0]->device) return fail(RD_ERR_ARG, "all detectors must be on one device");
    }
    rd_detector* d0 = dets[0];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // Segments (a problem's particles [p0, p0 + np)) in groups whose records fit the budget; each
    // group is one record precompute per segment and one persistent launch over its segments.
    struct Seg {
        int prob, p0, np, chunk;
        size_t rec_off;
    };
    std::vector<Seg> segs;
    std::vector<int> group_first{0};          // group g = segs[group_first[g], group_first[g + 1])
    std::vector<long long> item_off{0};       // per segment, restarting at 0 in every group
    size_t used = 0, rec_need = 256;
    // Step chunks: the persistent launch fills the GPU from all problems at once, so every problem
    // without a chunk of its own takes one batch-wide length: the default, halved (down to 512) while
    // the batch has fewer than kBatchItemsPerSm items per multiprocessor, since the items still
    // running at the end of the launch then leave much of the GPU idle (64 problems of 1-50
    // electrons: 53.3 ms at 4096-step chunks, 47.0 at 1024, 46.3 at 512).  A batch too small to
    // fill the GPU even so takes each problem's own choice.
    auto items_at = [&](int cap) {
        long long items = 0;
        for (int i = 0; i < n; ++i) {
            const int S = trajs[i].n_samples - 1;
            if (trajs[i].n_part == 0 || S < 1) continue;
            const int ncb = (dets[i]->n_pix + kMixedCellsPerCta - 1) / kMixedCellsPerCta;
            const int ck = dets[i]->chunk_override > 0 ? std::min(dets[i]->chunk_override, S) : std::min(cap, S);
            items += (long long)ncb * trajs[i].n_part * ((S + ck - 1) / ck);
        }
        return items;
    };
    int cap = kDefaultChunk;
    while (cap > 512 && items_at(cap) < (long long)kBatchItemsPerSm * sm_count()) cap /= 2;
    const bool full_chunks = items_at(cap) >= 8LL * sm_count();
    // problems of one walk family form consecutive groups: each group is one launch of its
    // family's persistent kernel
    auto family_of = [&](int i) {
        const int f = dets[i]->flags;
        return ((f & RD_FARFIELD) ? 4 : 0) + ((f & RD_QUADRATIC) ? 2 : (f & (RD_LINEAR | RD_HOLD_PREV)) ? 1 : 0);
    };
    std::vector<int> order;
    for (int fam : {0, 1, 2, 4, 5, 6})
        for (int i = 0; i < n; ++i)
            if (family_of(i) == fam) order.push_back(i);
    for (int i : order) {
        const rd_traj& t = trajs[i];
        const int S = t.n_samples - 1;
        if (t.n_part == 0 || S < 1) continue;
        if (!segs.empty() && family_of(segs.back().prob) != family_of(i) && group_first.back() != (int)segs.size()) {
            group_first.push_back((int)segs.size());            // a new family starts a new group
            item_off.push_back(0);
            used = 0;
        }
        const size_t per_part = sizeof(RecS) * (size_t)t.n_samples;
        const size_t budget = std::max(d0->batch_budget, per_part);
        const int ncb = (dets[i]->n_pix + kMixedCellsPerCta - 1) / kMixedCellsPerCta;
        const int chunk = full_chunks ? (dets[i]->chunk_override > 0 ? std::min(dets[i]->chunk_override, S)
                                                                      : std::min(cap, S))
                                      : choose_chunk(dets[i], t.n_part, S, ncb);
        for (int p0 = 0; p0 < t.n_part;) {
            if (budget - std::min(used, budget) < per_part && group_first.back() != (int)segs.size()) {
                group_first.push_back((int)segs.size());           // close the group
                item_off.push_back(0);
                used = 0;
            }
            // a segment's items are indexed in 32 bits by the kernel
            const long long per_p = (long long)ncb * ((S + chunk - 1) / chunk);
            const int np = (int)std::min<long long>(std::min<size_t>((size_t)(t.n_part - p0), (budget - used) / per_part),
                                                    std::max(1LL, 0x7fffffffLL / per_p));
            segs.push_back({i, p0, np, chunk, used});
            item_off.push_back(item_off.back() + (long long)ncb * np * ((S + chunk - 1) / chunk));
            used += per_part * np;
            rec_need = std::max(rec_need, used);
            p0 += np;
        }
    }
    const int n_seg = (int)segs.size();
    const int n_groups = n_seg ? (int)group_first.size() : 0;
    group_first.push_back(n_seg);
    // device tables: DepositParams[n_seg], item offsets (n_seg + n_groups), one counter per group
    const size_t off_bytes = sizeof(long long) * item_off.size();
    const size_t cnt_at = (sizeof(DepositParams) * n_seg + off_bytes + 15) & ~size_t(15);
    const size_t tab_bytes = cnt_at + sizeof(unsigned long long) * std::max(1, n_groups);
    rd_status st = ensure(&d0->batch_rec, &d0->batch_rec_bytes, rec_need, s, "batch records");
    if (st != RD_OK) return st;
    st = ensure(&d0->batch_tab, &d0->batch_tab_bytes, tab_bytes, s, "batch table");
    if (st != RD_OK) return st;
    char* tab = static_cast<char*>(d0->batch_tab);
    DepositParams* d_probs = reinterpret_cast<DepositParams*>(tab);
    long long* d_off = reinterpret_cast<long long*>(tab + sizeof(DepositParams) * n_seg);
    unsigned long long* d_counter = reinterpret_cast<unsigned long long*>(tab + cnt_at);
    // graph key: everything a replay depends on
    std::vector<unsigned long long> key;
    key.push_back((unsigned long long)n);
    key.push_back((unsigned long long)(uintptr_t)d0->batch_rec);
    key.push_back((unsigned long long)(uintptr_t)d0->batch_tab);
    key.push_back((unsigned long long)(uintptr_t)s);
    key.push_back((unsigned long long)d0->batch_budget);
    for (int i = 0; i < n; ++i) {
        const rd_traj& t = trajs[i];
        unsigned long long t0b, dtb;
        memcpy(&t0b, &t.t0, 8);
        memcpy(&dtb, &t.dt, 8);
        key.insert(key.end(), {dets[i]->id, (unsigned long long)(uintptr_t)t.x, (unsigned long long)(uintptr_t)t.u,
                               (unsigned long long)(uintptr_t)t.q, (unsigned long long)t.n_part,
                               (unsigned long long)t.n_samples, t0b, dtb, (unsigned long long)dets[i]->flags,
                               (unsigned long long)dets[i]->chunk_override});
    }
    const bool reuse = d0->graph_exec && key == d0->graph_key;
    if (!reuse && n_seg > 0) {
        // segment table (stays in device memory for replays)
        std::vector<DepositParams> probs(n_seg);
        for (int k = 0; k < n_seg; ++k) {
            const Seg& g = segs[k];
            const rd_traj& t = trajs[g.prob];
            const size_t off = (size_t)g.p0 * t.n_samples * 3;
            fill_mixed_params(probs[k], dets[g.prob], &t, static_cast<char*>(d0->batch_rec) + g.rec_off, t.x + off,
                              t.q ? t.q + g.p0 : nullptr, g.np, g.chunk);
        }
        RD_CUDA(cudaMemcpyAsync(d_probs, probs.data(), sizeof(DepositParams) * n_seg, cudaMemcpyHostToDevice, s),
                "batch table");
        RD_CUDA(cudaMemcpyAsync(d_off, item_off.data(), off_bytes, cudaMemcpyHostToDevice, s), "batch table");
        RD_CUDA(cudaStreamSynchronize(s), "batch table");     // host vectors go out of scope
    }
    if (!reuse && d0->graph_exec) {
        cudaGraphExecDestroy(d0->graph_exec);
        d0->graph_exec = nullptr;
    }
    auto enqueue = [&]() -> cudaError_t {
        if (n_seg == 0) return cudaSuccess;
        cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long) * n_groups, s);
        for (int gi = 0; gi < n_groups && e == cudaSuccess; ++gi) {
            const int a = group_first[gi], b = group_first[gi + 1];
            for (int k = a; k < b && e == cudaSuccess; ++k) {
                const Seg& g = segs[k];
                const rd_traj& t = trajs[g.prob];
                const size_t off = (size_t)g.p0 * t.n_samples * 3;
                e = launch_precompute_mixed(t.x + off, t.u + off, t.q ? t.q + g.p0 : nullptr, t.dt / dets[g.prob]->dt_det,
                                            g.np, t.n_samples, t.dt, dets[g.prob]->flags,
                                            reinterpret_cast<RecS*>(static_cast<char*>(d0->batch_rec) + g.rec_off),
                                            dets[g.prob]->counters, s);
            }
            // segment k's items are d_off[k + gi], relative to the group's first item
            if (e == cudaSuccess)
                e = launch_deposit_batch(family_of(segs[a].prob), d_probs + a, d_off + a + gi, b - a, d_counter + gi, s);
        }
        return e;
    };
    if (s == nullptr) {
        // the legacy default stream cannot be captured: launch directly
        RD_CUDA(enqueue(), "rd_deposit_batch");
    } else if (n_seg > 0) {
        if (!reuse) {
            cudaGraph_t graph = nullptr;
            RD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture batch");
            const cudaError_t e = enqueue();
            const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(e != cudaSuccess ? e : e2, "capture batch");
            }
            const cudaError_t e3 = cudaGraphInstantiate(&d0->graph_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e3 != cudaSuccess) {
                d0->graph_exec = nullptr;
                return cuda_fail(e3, "instantiate batch graph");
            }
            d0->graph_key = key;
        }
        LaunchTimer timer(d0, s);
        RD_CUDA(cudaGraphLaunch(d0->graph_exec, s), "launch batch graph");
    }
    for (int i = 0; i < n; ++i)
        dets[i]->n_deposits += (long long)trajs[i].n_part * std::max(0, trajs[i].n_samples - 1) * dets[i]->n_pix;
    return RD_OK;
}

rd_status rd_power_spectrum(rd_detector* d, int32_t which, float* out, rd_stream stream)
{
    g_err.clear();
    if (!d || !out) return fail(RD_ERR_ARG, "detector/out is NULL");
    if (which != RD_SPEC_E && which != RD_SPEC_B) return fail(RD_ERR_ARG, "bad field selector %d", which);
    const int N = d->n_bins;
    if (N < 2 || (N & (N - 1)) != 0) return fail(RD_ERR_ARG, "n_bins must be a power of two >= 2 (got %d)", N);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // work arrays for the pass-per-launch transform of long series (none for the fused one)
    const size_t work = spectrum_fused(N) ? 0 : sizeof(float2) * 2 * (size_t)d->n_pix * N;
    rd_status st = work ? ensure(&d->spec, &d->spec_bytes, 2 * work, s, "spectrum scratch") : RD_OK;
    if (st != RD_OK) return st;
    if (d->spec_n != N) {
        st = ensure(&d->spec_tw, &d->spec_tw_bytes, sizeof(float2) * (N / 2), s, "twiddles");
        if (st != RD_OK) return st;
        RD_CUDA(cudaStreamSynchronize(s), "twiddles");          // the host table may be in flight
        d->spec_tw_host.resize(N / 2);
        fill_twiddles(d->spec_tw_host.data(), N);
        RD_CUDA(cudaMemcpyAsync(d->spec_tw, d->spec_tw_host.data(), sizeof(float2) * (N / 2), cudaMemcpyHostToDevice,
                                s),
                "twiddles");
        d->spec_n = N;
    }
    float2* z = work ? static_cast<float2*>(d->spec) : nullptr;
    float2* y = work ? reinterpret_cast<float2*>(static_cast<char*>(d->spec) + work) : nullptr;
    RD_CUDA(launch_power_spectrum(d->fields, d->precision, d->n_pix, N, which == RD_SPEC_B ? 3 : 0, z, y,
                                  static_cast<const float2*>(d->spec_tw), (float)(d->dt_det * d->dt_det), out, s),
            "power spectrum");
    return RD_OK;
}

rd_status rd_deposit_stream(rd_detector* d, const rd_traj* t, rd_stream stream)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    rd_status st = check_traj(t);
    if (st != RD_OK) return st;
    if (t->n_part < 1) return fail(RD_ERR_ARG, "a streamed call needs n_part >= 1");
    const bool cont = d->strm_n_part >= 0;
    if (cont) {
        if (t->n_part != d->strm_n_part)
            return fail(RD_ERR_STATE, "streamed call has %d particles, the stream %d (rd_stream_reset starts a new one)",
                        t->n_part, d->strm_n_part);
        if (fabs(t->dt - d->strm_dt) > 1e-12 * d->strm_dt)
            return fail(RD_ERR_STATE, "streamed call has dt = %.17g, the stream %.17g", t->dt, d->strm_dt);
        const double expect = d->strm_t_last + d->strm_dt;
        if (fabs(t->t0 - expect) > 1e-6 * t->dt + 1e-12 * fabs(expect))
            return fail(RD_ERR_STATE, "streamed call starts at t0 = %.17g, the stream continues at %.17g", t->t0,
                        expect);
    }
    // samples kept between calls: the last one (its interval to the first new sample), with RD_LINEAR /
    // RD_HOLD_PREV the one before it too (the field of the last sample needs its betadot), and with
    // RD_QUADRATIC one more (the field two samples back)
    const int keep = (d->flags & RD_QUADRATIC) ? 3 : (d->flags & (RD_LINEAR | RD_HOLD_PREV)) ? 2 : 1;
    const int have = cont ? d->strm_have : 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int np = t->n_part, m = t->n_samples, ns = m + have;
    const size_t one = 3 * sizeof(double);
    const size_t row = one * (size_t)ns, mrow = one * (size_t)m;
    st = ensure(&d->strm_stage, &d->strm_stage_bytes, 2 * row * np + sizeof(double) * np, s, "stream staging");
    if (st != RD_OK) return st;
    if (!cont) {
        st = ensure(&d->strm_last, &d->strm_last_bytes, 2 * one * 3 * np, s, "stream state");
        if (st != RD_OK) return st;
    }
    double* xs = static_cast<double*>(d->strm_stage);
    double* us = xs + (size_t)np * ns * 3;
    double* qs = us + (size_t)np * ns * 3;
    double* lx = static_cast<double*>(d->strm_last);        // [np][have][3], have <= 3
    double* lu = lx + (size_t)np * 3 * 3;
    const cudaMemcpyKind kind = t->mem == RD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    RD_CUDA(cudaMemcpy2DAsync(xs + 3 * have, row, t->x, mrow, mrow, np, kind, s), "stream x");
    RD_CUDA(cudaMemcpy2DAsync(us + 3 * have, row, t->u, mrow, mrow, np, kind, s), "stream u");
    if (have > 0) {
        RD_CUDA(cudaMemcpy2DAsync(xs, row, lx, one * have, one * have, np, cudaMemcpyDeviceToDevice, s), "stream x");
        RD_CUDA(cudaMemcpy2DAsync(us, row, lu, one * have, one * have, np, cudaMemcpyDeviceToDevice, s), "stream u");
    }
    if (t->q) RD_CUDA(cudaMemcpyAsync(qs, t->q, sizeof(double) * np, kind, s), "stream q");
    rd_traj staged = *t;
    staged.n_samples = ns;
    staged.x = xs;
    staged.u = us;
    staged.q = t->q ? qs : nullptr;
    staged.mem = RD_MEM_DEVICE;
    staged.t0 = t->t0 - have * t->dt;
    // intervals already deposited by earlier calls are not deposited again; the staged sample 0 is
    // sample strm_count - have of the whole trajectory
    const long long count0 = cont ? d->strm_count : 0;
    st = deposit_from(d, &staged, stream, std::max(1, have), (int)std::min<long long>(count0 - have, 1 << 30));
    if (st != RD_OK) return st;
    const int kept = std::min(keep, ns);
    RD_CUDA(cudaMemcpy2DAsync(lx, one * kept, xs + 3 * (size_t)(ns - kept), row, one * kept, np,
                              cudaMemcpyDeviceToDevice, s),
            "stream state");
    RD_CUDA(cudaMemcpy2DAsync(lu, one * kept, us + 3 * (size_t)(ns - kept), row, one * kept, np,
                              cudaMemcpyDeviceToDevice, s),
            "stream state");
    d->strm_n_part = np;
    d->strm_have = kept;
    d->strm_count = count0 + m;
    d->strm_t_last = t->t0 + (double)(m - 1) * t->dt;
    d->strm_dt = t->dt;
    return RD_OK;
}

rd_status rd_stream_reset(rd_detector* d)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    d->strm_n_part = -1;
    return RD_OK;
}

rd_status rd_set_batch_budget(rd_detector* d, long long bytes)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    if (bytes < 0) return fail(RD_ERR_ARG, "budget must be >= 0 (got %lld)", bytes);
    d->batch_budget = bytes > 0 ? (size_t)bytes : kBatchBudgetDefault;
    return RD_OK;
}

rd_status rd_set_timing(rd_detector* d, int32_t enable)
{
    g_err.clear();
    if (!d) return fail(RD_ERR_ARG, "detector is NULL");
    d->timing = enable != 0;
    return RD_OK;
}

}  // extern "C"
