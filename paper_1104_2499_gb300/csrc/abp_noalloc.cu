// abp_noalloc.cu -- abp_run_set_noalloc: one parameter set integrated and
// reduced without any device allocation.
//
// Some callers cannot allocate device memory themselves or let a library do
// it: code running under a host framework that owns all device memory through
// its own pool and forbids cudaMalloc / cudaFree (which also synchronise the
// device), or a latency-critical loop that must never stall on an allocation.
// For them this entry point keeps every piece of scratch memory the run needs
// (trajectory state, tile table, reduction partials) in one file-scope
// __device__ array of fixed size, reserved when the library is loaded; the
// caller passes only the outputs.  The kernels are the same ones the
// context-based entry points use.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "abp.h"
#include "abp_device.cuh"
#include "abp_internal.cuh"

namespace abp {
namespace {

// Largest ensemble the static scratch holds.
constexpr int64_t kNoAllocMaxTraj = ABP_NOALLOC_MAX_TRAJ;
constexpr int64_t kNoAllocMaxTiles = kNoAllocMaxTraj / kThreads;  // tiles hold >= kThreads trajectories

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets inside the scratch array.
constexpr size_t kOffY = 0;
constexpr size_t kOffYacc = kOffY + align256(sizeof(float) * kNoAllocMaxTraj);
constexpr size_t kOffYlo = kOffYacc + align256(sizeof(float) * kNoAllocMaxTraj);
constexpr size_t kOffV = kOffYlo + align256(sizeof(float) * kNoAllocMaxTraj);
constexpr size_t kOffE = kOffV + align256(sizeof(float) * kNoAllocMaxTraj);
constexpr size_t kOffY0 = kOffE + align256(sizeof(float) * kNoAllocMaxTraj);
constexpr size_t kOffCell = kOffY0 + align256(sizeof(float) * kNoAllocMaxTraj);
constexpr size_t kOffPartials = kOffCell + align256(sizeof(int32_t) * kNoAllocMaxTraj);
constexpr size_t kOffParams = kOffPartials + align256(sizeof(double) * 4 * kNoAllocMaxTiles);
constexpr size_t kOffSteps = kOffParams + align256(sizeof(abp_params));
constexpr size_t kOffSetTiles = kOffSteps + align256(sizeof(int64_t));
constexpr size_t kOffTileFirst = kOffSetTiles + align256(sizeof(int32_t) * 2);
constexpr size_t kOffTileCount = kOffTileFirst + align256(sizeof(int64_t) * kNoAllocMaxTiles);
constexpr size_t kOffTileSet = kOffTileCount + align256(sizeof(int32_t) * kNoAllocMaxTiles);
constexpr size_t kScratchBytes = kOffTileSet + align256(sizeof(int32_t) * kNoAllocMaxTiles);
static_assert(kScratchBytes == ABP_NOALLOC_SCRATCH_BYTES, "header states the scratch size");

// The scratch itself: every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Tile table and parameters of the single set, written on the device from
// kernel arguments (device code names the array directly).
__global__ void noalloc_tables_kernel(abp_params p, int64_t n_traj, int64_t n_steps, int32_t tile, int32_t n_tiles) {
    unsigned char *base = g_noalloc_scratch;
    if (threadIdx.x == 0) {
        *(abp_params *)(base + kOffParams) = p;
        *(int64_t *)(base + kOffSteps) = n_steps;
        int32_t *st = (int32_t *)(base + kOffSetTiles);
        st[0] = 0;
        st[1] = n_tiles;
    }
    int64_t *first = (int64_t *)(base + kOffTileFirst);
    int32_t *count = (int32_t *)(base + kOffTileCount);
    int32_t *set = (int32_t *)(base + kOffTileSet);
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const int64_t f = (int64_t)t * tile;
        first[t] = f;
        count[t] = (int32_t)(n_traj - f < tile ? n_traj - f : tile);
        set[t] = 0;
    }
}

// Device address of the scratch array, looked up once per device with that
// device current (a host-side reference to the symbol is not a device address).
std::mutex g_addr_mu;
constexpr int kMaxDevices = 64;
void *g_addr[kMaxDevices] = {};

cudaError_t scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = (unsigned char *)g_addr[dev];
    return cudaSuccess;
}

abp_status say(char *err, size_t err_len, abp_status st, const char *fmt, ...) {
    if (err && err_len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, err_len, fmt, ap);
        va_end(ap);
    }
    return st;
}

// The outputs are written by kernels on the current device: they must be that
// device's memory (or managed memory), not host memory nor another GPU's.
bool on_device(const void *p, int dev) { return ptr_kind(p, dev) == PtrKind::Device; }

}  // namespace
}  // namespace abp

using namespace abp;

extern "C" abp_status abp_run_set_noalloc(const abp_params *params, const abp_config *cfg, int64_t n_traj,
                                          int64_t n_steps, double *moments, uint32_t *hist_x, uint32_t *hist_v,
                                          void *cuda_stream, char *err, size_t err_len) {
    if (err && err_len) err[0] = '\0';
    if (!params || !cfg) return say(err, err_len, ABP_EINVAL, "params and cfg must not be NULL");
    const abp_params &p = *params;
    const double pv[9] = {p.q, p.c, p.d, p.gamma0, p.F0, p.D, p.h, p.L, p.asym};
    for (double x : pv)
        if (!std::isfinite(x)) return say(err, err_len, ABP_EINVAL, "non-finite parameter");
    if (!(p.L > 0.0)) return say(err, err_len, ABP_EINVAL, "L = %g must be > 0", p.L);
    if (p.D < 0.0) return say(err, err_len, ABP_EINVAL, "D = %g must be >= 0", p.D);
    if (!(cfg->dt > 0.0) || !std::isfinite(cfg->dt)) return say(err, err_len, ABP_EINVAL, "dt must be > 0");
    if (cfg->v0_mode != 0 && cfg->v0_mode != 1) return say(err, err_len, ABP_EINVAL, "v0_mode must be 0 or 1");
    if (cfg->state_fp64 != 0)
        return say(err, err_len, ABP_EINVAL, "the allocation-free entry point runs the FP32 state only");
    if (cfg->checkpoint_every != 0)
        return say(err, err_len, ABP_EINVAL, "the allocation-free entry point keeps no adjoint checkpoints");
    if (cfg->hist_x_bins < 0 || cfg->hist_v_bins < 0 || cfg->hist_x_bins > 8192 || cfg->hist_v_bins > 8192)
        return say(err, err_len, ABP_EINVAL, "histogram bins must be in [0, 8192]");
    if (cfg->hist_v_bins > 0 && !(cfg->v_hi > cfg->v_lo))
        return say(err, err_len, ABP_EINVAL, "v_hi must exceed v_lo");
    if (cfg->scheme != 0 && cfg->scheme != 1) return say(err, err_len, ABP_EINVAL, "scheme must be 0 or 1");
    if (cfg->noise != 0)
        return say(err, err_len, ABP_EINVAL, "the allocation-free entry point uses the counter-based noise only");
    if (cfg->snapshot_every < 0 || cfg->steps_per_launch < 0)
        return say(err, err_len, ABP_EINVAL, "invalid snapshot_every / steps_per_launch");
    // the work queue needs per-tile counters and an autotuner table, which this call has no
    // room for: it always runs lockstep launches of one block per tile
    if (cfg->schedule != 0 && cfg->schedule != 1)
        return say(err, err_len, ABP_EINVAL,
                   "schedule = %d: the allocation-free entry point runs the lockstep schedule only (0 or 1)",
                   cfg->schedule);
    const int ppt = cfg->particles_per_thread ? cfg->particles_per_thread : 1;
    if (ppt != 1 && ppt != 2 && ppt != 4) return say(err, err_len, ABP_EINVAL, "particles_per_thread must be 1, 2 or 4");
    if (n_traj < 0 || n_traj > kNoAllocMaxTraj)
        return say(err, err_len, ABP_EINVAL,
                   "n_traj = %lld is outside [0, %lld], the capacity of the static scratch (use abp_create for "
                   "larger ensembles)",
                   (long long)n_traj, (long long)kNoAllocMaxTraj);
    if (n_steps < 0 || n_steps >= ((int64_t)1 << 34))
        return say(err, err_len, ABP_EINVAL, "n_steps must be in [0, 2^34)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return say(err, err_len, ABP_ECUDA, "no current device: %s", cudaGetErrorString(e));
    if (!moments || !on_device(moments, dev))
        return say(err, err_len, ABP_EINVAL, "moments must be memory of the current device (%d)", dev);
    if (cfg->hist_x_bins > 0 && (!hist_x || !on_device(hist_x, dev)))
        return say(err, err_len, ABP_EINVAL, "hist_x must be memory of the current device when hist_x_bins > 0");
    if (cfg->hist_v_bins > 0 && (!hist_v || !on_device(hist_v, dev)))
        return say(err, err_len, ABP_EINVAL, "hist_v must be memory of the current device when hist_v_bins > 0");

    unsigned char *base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess) return say(err, err_len, ABP_ECUDA, "scratch set-up: %s", cudaGetErrorString(e));

    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int32_t tile = kThreads * ppt;
    const int32_t n_tiles = (int32_t)((n_traj + tile - 1) / tile);
    const bool any_hist = cfg->hist_x_bins > 0 || cfg->hist_v_bins > 0;
    const int64_t n_snap = any_hist ? (cfg->snapshot_every > 0 ? n_steps / cfg->snapshot_every : 1) : 0;

    // Outputs the kernels accumulate into start at zero.
    if (cfg->hist_x_bins > 0 && n_snap > 0)
        e = cudaMemsetAsync(hist_x, 0, sizeof(uint32_t) * (size_t)n_snap * cfg->hist_x_bins, st);
    if (e == cudaSuccess && cfg->hist_v_bins > 0 && n_snap > 0)
        e = cudaMemsetAsync(hist_v, 0, sizeof(uint32_t) * (size_t)n_snap * (cfg->hist_v_bins + 2), st);
    if (e != cudaSuccess) return say(err, err_len, ABP_ECUDA, "histogram clear: %s", cudaGetErrorString(e));

    noalloc_tables_kernel<<<1, kThreads, 0, st>>>(p, n_traj, n_steps, tile, n_tiles);

    Batch b;
    b.n_sets = 1;
    b.n_tiles = n_tiles;
    b.n_single = n_tiles;
    b.set_first = nullptr;
    b.set_order = nullptr;
    b.slot_set = nullptr;
    b.n_unpacked = b.n_sets;
    b.narrow = 0;
    b.sub_single = b.sub_packed = 1;
    b.total_traj = n_traj;
    b.params = (const abp_params *)(base + kOffParams);
    b.set_steps = (const int64_t *)(base + kOffSteps);
    b.set_tile_begin = (const int32_t *)(base + kOffSetTiles);
    b.tile_first = (const int64_t *)(base + kOffTileFirst);
    b.tile_count = (const int32_t *)(base + kOffTileCount);
    b.tile_set = (const int32_t *)(base + kOffTileSet);
    State s;
    s.fp64 = false;
    s.y = base + kOffY;
    s.yacc = base + kOffYacc;
    s.ylo = base + kOffYlo;
    s.v = base + kOffV;
    s.e = base + kOffE;
    s.y0 = base + kOffY0;
    s.cell = (int32_t *)(base + kOffCell);
    s.xs = nullptr;
    Hist h;
    h.x = hist_x;
    h.v = hist_v;
    h.bx = cfg->hist_x_bins;
    h.bv = cfg->hist_v_bins;
    h.v_lo = cfg->v_lo;
    h.v_hi = cfg->v_hi;
    h.snap_every = cfg->snapshot_every;
    h.n_snap = n_snap;
    Ckpt c;
    c.ck = nullptr;
    c.every = 0;
    c.n_slots = 0;
    Noise nz;
    memset(&nz, 0, sizeof(nz));
    nz.k0 = (uint32_t)cfg->seed;
    nz.k1 = (uint32_t)(cfg->seed >> 32);
    nz.dt = cfg->dt;
    nz.v0_mode = cfg->v0_mode;
    nz.traj_base = cfg->traj_base;
    nz.scheme = cfg->scheme;
    nz.noise = 0;

    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_init(b, s, h, c, nz, st);
    const int64_t spl = cfg->steps_per_launch > 0 ? cfg->steps_per_launch : (n_steps > 0 ? n_steps : 1);
    for (int64_t g = 0; e == cudaSuccess && g < n_steps; g += spl)
        e = launch_integrate(b, s, h, c, nz, ppt, g, g + spl < n_steps ? g + spl : n_steps, st);
    if (e == cudaSuccess) e = launch_reduce(b, s, nz, n_steps, (double *)(base + kOffPartials), moments, st);
    if (e != cudaSuccess) return say(err, err_len, ABP_ECUDA, "launch: %s", cudaGetErrorString(e));
    return ABP_OK;
}
