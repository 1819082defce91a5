// Allocation-free form of the mixed-precision deposit.
//
// Some callers cannot call cudaMalloc.  A particle-in-cell code typically reserves its device
// memory in its own pool at start-up and does not allow further allocations inside its time-step
// loop.  A host framework may own all device memory through its own allocator.  And a latency-bound
// loop must not pay the device-wide synchronisation that cudaMalloc and cudaFree can cause.
// rd_deposit_noalloc serves these callers.  It runs the same precompute and deposit kernels as
// rd_deposit_trajectories on an RD_MIXED detector, but needs no rd_detector object.  The caller
// passes the inputs and the output accumulators.  All scratch (per-sample records, the cell table
// and the error counters) comes from one file-scope device array of fixed size, kNoallocBytes.
// Every GPU that loads this library holds that array until the process exits.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "rd_internal.cuh"

namespace rd {

rd_status set_last_error(rd_status st, const char* msg);   // rd_api.cu

namespace {

constexpr size_t kNoallocBytes = size_t(64) << 20;                  // 64 MiB in all
constexpr int kNoallocMaxCells = 262144;                             // cell table: 8 MiB
constexpr size_t kCounterBytes = 256;
constexpr size_t kCellBytes = sizeof(D4) * (size_t)kNoallocMaxCells;
constexpr size_t kRecordBytes = kNoallocBytes - kCounterBytes - kCellBytes;   // ~56 MiB

static __device__ __align__(256) unsigned char rd_noalloc_scratch[kNoallocBytes];

std::mutex g_setup_mu;
constexpr int kMaxDevices = 256;
void* g_scratch[kMaxDevices] = {};   // device address of rd_noalloc_scratch, per device

// Device address of the scratch array on the current device, looked up on the first call there.
rd_status scratch_address(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_last_error(RD_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_last_error(RD_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, rd_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
            return set_last_error(RD_ERR_CUDA, msg);
        }
        g_scratch[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch[dev]);
    return RD_OK;
}

// cell table (x, y, z, T0 = t_min + pix_t0) from the caller's arrays; a cell with a non-finite
// position or time origin latches ERRBIT_INPUT (the call's deposits are then undefined)
__global__ void k_cell_table(const double* __restrict__ pos, const double* __restrict__ t0, int n, double t_min,
                             D4* __restrict__ cells, DevCounters* counters)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const D4 c{pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], t_min + (t0 ? t0[j] : 0.0)};
        if (!isfinite(c.x) || !isfinite(c.y) || !isfinite(c.z) || !isfinite(c.w))
            atomicOr(&counters->errors, ERRBIT_INPUT);
        cells[j] = c;
    }
}

}  // namespace
}  // namespace rd

using namespace rd;

extern "C" rd_status rd_deposit_noalloc(const double* pix_pos, const double* pix_t0, int32_t n_pix, double t_min,
                                        double dt_det, int32_t n_bins, int32_t flags, const rd_traj* t,
                                        float* fields, uint32_t* errors, rd_stream stream)
{
    set_last_error(RD_OK, "");
    if (!pix_pos || !fields || !t) return set_last_error(RD_ERR_ARG, "pix_pos, fields and traj must be given");
    if (n_pix < 1 || n_bins < 1) return set_last_error(RD_ERR_ARG, "n_pix and n_bins must be >= 1");
    if (n_bins > kMixedMaxBins) return set_last_error(RD_ERR_ARG, "n_bins must be <= 4194304");
    if (n_pix > kNoallocMaxCells)
        return set_last_error(RD_ERR_ARG, "rd_deposit_noalloc: n_pix exceeds its maximum of 262144 cells");
    if (!(dt_det > 0.0) || !isfinite(dt_det) || !isfinite(t_min))
        return set_last_error(RD_ERR_ARG, "dt_det must be finite and > 0, t_min finite");
    if (const char* why = flags_error(flags)) return set_last_error(RD_ERR_ARG, why);
    if (t->n_part < 0 || t->n_samples < 1 || !(t->dt > 0.0) || !isfinite(t->dt) || !isfinite(t->t0))
        return set_last_error(RD_ERR_ARG, "bad trajectory shape or time axis");
    if (t->mem != RD_MEM_DEVICE) return set_last_error(RD_ERR_ARG, "rd_deposit_noalloc needs device trajectories");
    if (t->n_part > 0 && (!t->x || !t->u)) return set_last_error(RD_ERR_ARG, "traj x/u is NULL");
    const size_t per_part = sizeof(RecS) * (size_t)t->n_samples;
    if (per_part > kRecordBytes)
        return set_last_error(RD_ERR_ARG, "rd_deposit_noalloc: one particle's samples exceed the 56 MiB record scratch "
                                          "(at most 917500 samples per particle)");
    unsigned char* base = nullptr;
    rd_status st = scratch_address(&base);
    if (st != RD_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevCounters* counters = reinterpret_cast<DevCounters*>(base);
    D4* cells = reinterpret_cast<D4*>(base + kCounterBytes);
    RecS* records = reinterpret_cast<RecS*>(base + kCounterBytes + kCellBytes);
    const int fl = flags ? flags : (RD_NEAR | RD_FAR);

    // the array keeps the previous call's contents: counters must start at zero
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(DevCounters), s);
    if (e == cudaSuccess) {
        k_cell_table<<<(n_pix + 255) / 256, 256, 0, s>>>(pix_pos, pix_t0, n_pix, t_min, cells, counters);
        e = cudaGetLastError();
    }
    const int S = t->n_samples - 1;
    if (e == cudaSuccess && t->n_part > 0 && S >= 1) {
        const int pc = (int)std::max<size_t>(1, std::min<size_t>((size_t)t->n_part, kRecordBytes / per_part));
        const int n_cell_blocks = (n_pix + kMixedCellsPerCta - 1) / kMixedCellsPerCta;
        const int chunk = auto_chunk(n_cell_blocks, std::min(pc, t->n_part), S);
        for (int p0 = 0; p0 < t->n_part && e == cudaSuccess; p0 += pc) {
            const int np = std::min(pc, t->n_part - p0);
            const size_t off = (size_t)p0 * t->n_samples * 3;
            e = launch_precompute_mixed(t->x + off, t->u + off, t->q ? t->q + p0 : nullptr, t->dt / dt_det, np,
                                        t->n_samples, t->dt, fl, records, counters, s);
            if (e != cudaSuccess) break;
            DepositParams P;
            P.rec = records;
            P.x = t->x + off;
            P.q = t->q ? t->q + p0 : nullptr;
            P.cells = cells;
            P.fields = fields;
            P.counters = counters;
            P.n_pix = n_pix;
            P.n_bins = n_bins;
            P.n_samples = t->n_samples;
            P.n_part = np;
            P.chunk = chunk;
            P.k_first = 1;
            P.n_chunks = (S + chunk - 1) / chunk;
            P.n_cell_blocks = n_cell_blocks;
            P.t0 = t->t0;
            P.dt = t->dt;
            P.inv_dt_det = 1.0 / dt_det;
            P.dt_f = (float)t->dt;
            P.du_scale = (float)(t->dt / dt_det);
            P.W = (float)(dt_det / t->dt);
            P.invW = (float)(t->dt / dt_det);
            P.ff = (fl & RD_FARFIELD) != 0;
            P.lin = (fl & RD_LINEAR) ? 1 : (fl & RD_HOLD_PREV) ? 2 : (fl & RD_QUADRATIC) ? 3 : 0;
            P.group = cell_group(n_cell_blocks, n_bins, kMixedCellsPerCta, chunk, S);
            e = launch_deposit_mixed(P, s);
        }
    }
    if (e != cudaSuccess) return set_last_error(RD_ERR_CUDA, cudaGetErrorString(e));
    if (errors) {
        DevCounters c;
        e = cudaMemcpyAsync(&c, counters, sizeof c, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_last_error(RD_ERR_CUDA, cudaGetErrorString(e));
        *errors = c.errors;
    }
    return RD_OK;
}
