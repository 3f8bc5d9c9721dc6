// abp_api.cu -- host runtime of the C ABI declared in include/abp.h.
//
// Owns the device buffers of a batch (structure-of-arrays trajectory state,
// tile table, histograms, adjoint checkpoints, reduction scratch), validates
// every argument, tiles the parameter sets for the device and enqueues the
// kernels of abp_kernels.cu / abp_adjoint.cu on the context's stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "abp.h"
#include "abp_ctx.cuh"
#include "abp_internal.cuh"

using namespace abp;

namespace {

abp_status fail(abp_ctx *ctx, abp_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return st;
}

abp_status cuda_fail(abp_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? ABP_ENOMEM : ABP_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

#define ABP_CUDA(ctx, call, what)                      \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

// Size b for `bytes`, reusing its allocation when the capacity suffices.
abp_status alloc(abp_ctx *ctx, DevBuf &b, size_t bytes, const char *what) {
    if (b.p && b.cap >= bytes) {
        b.bytes = bytes;
        return ABP_OK;
    }
    b.release();
    if (bytes == 0) return ABP_OK;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(ctx, ABP_ENOMEM, "cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
    }
    b.cap = bytes;
    b.bytes = bytes;
    return ABP_OK;
}

// True if ptr is device-accessible memory (device or managed); false for host
// memory (pinned or pageable).
bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool finite_params(const abp_params &p) {
    const double v[9] = {p.q, p.c, p.d, p.gamma0, p.F0, p.D, p.h, p.L, p.asym};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

int64_t default_steps_per_launch(const abp_ctx *ctx) {
    // About 2e10 particle-steps per launch (tens of ms on a GB300), a multiple of 64.
    if (ctx->total_traj == 0) return std::max<int64_t>(ctx->max_steps, 1);
    int64_t s = (int64_t)(2.0e10 / (double)ctx->total_traj);
    s = std::max<int64_t>(64, (s / 64) * 64);
    return std::max<int64_t>(1, std::min<int64_t>(s, std::max<int64_t>(ctx->max_steps, 1)));
}

// Copy n bytes of a device buffer to a caller pointer that may be host or device.
abp_status deliver(abp_ctx *ctx, void *dst, const void *src, size_t n, bool *synced) {
    if (!dst || n == 0) return ABP_OK;
    if (is_device_ptr(dst)) {
        ABP_CUDA(ctx, cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, ctx->stream), "copy to device output");
    } else {
        ABP_CUDA(ctx, cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, ctx->stream), "copy to host output");
        *synced = true;
    }
    return ABP_OK;
}

}  // namespace

// ====================================================================== ABI

extern "C" {

const char *abp_version(void) { return "abp-gb300 1.0 (sm_103a)"; }

const char *abp_last_error(const abp_ctx *ctx) {
    if (!ctx) return "abp: NULL context";
    return ctx->err.c_str();
}

abp_status abp_create(abp_ctx **out, const abp_config *cfg, void *cuda_stream) {
    if (!out || !cfg) return ABP_EINVAL;
    *out = nullptr;
    if (!(cfg->dt > 0.0) || !std::isfinite(cfg->dt)) return ABP_EINVAL;
    if (cfg->v0_mode != 0 && cfg->v0_mode != 1) return ABP_EINVAL;
    if (cfg->state_fp64 != 0 && cfg->state_fp64 != 1) return ABP_EINVAL;
    if (cfg->hist_x_bins < 0 || cfg->hist_v_bins < 0 || cfg->hist_x_bins > 8192 || cfg->hist_v_bins > 8192)
        return ABP_EINVAL;
    if (cfg->hist_v_bins > 0 && !(cfg->v_hi > cfg->v_lo && std::isfinite(cfg->v_lo) && std::isfinite(cfg->v_hi)))
        return ABP_EINVAL;
    if (cfg->snapshot_every < 0 || cfg->checkpoint_every < 0 || cfg->steps_per_launch < 0) return ABP_EINVAL;
    if (cfg->particles_per_thread != 0 && cfg->particles_per_thread != 1 && cfg->particles_per_thread != 2 &&
        cfg->particles_per_thread != 4)
        return ABP_EINVAL;
    if (cfg->reserved != 0) return ABP_EINVAL;
    if (cfg->checkpoint_every > 0 && cfg->state_fp64) return ABP_EINVAL;  // adjoint runs on the FP32 path
    abp_ctx *ctx = new (std::nothrow) abp_ctx();
    if (!ctx) return ABP_ENOMEM;
    ctx->cfg = *cfg;
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) {
        e = cudaMalloc(&ctx->d_status.p, sizeof(int32_t));
        if (e == cudaSuccess) {
            ctx->d_status.cap = ctx->d_status.bytes = sizeof(int32_t);
            e = cudaMemsetAsync(ctx->d_status.p, 0, sizeof(int32_t), ctx->stream);
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->d_status.release();
        delete ctx;
        return e == cudaErrorMemoryAllocation ? ABP_ENOMEM : ABP_ECUDA;
    }
    ctx->ppt = cfg->particles_per_thread ? cfg->particles_per_thread : 1;
    *out = ctx;
    return ABP_OK;
}

void abp_destroy(abp_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    ctx->release_all();
    ctx->d_status.release();
    delete ctx;
}

abp_status abp_set_params(abp_ctx *ctx, int32_t n_sets, const abp_params *sets, const int64_t *n_traj,
                          const int64_t *n_steps) {
    if (!ctx) return ABP_EINVAL;
    if (n_sets < 0) return fail(ctx, ABP_EINVAL, "n_sets = %d < 0", n_sets);
    if (n_sets > 0 && (!sets || !n_traj || !n_steps)) return fail(ctx, ABP_EINVAL, "NULL parameter array");
    int64_t total = 0, max_n = 0;
    for (int32_t i = 0; i < n_sets; ++i) {
        const abp_params &p = sets[i];
        if (!finite_params(p)) return fail(ctx, ABP_EINVAL, "set %d: non-finite parameter", i);
        if (!(p.L > 0.0)) return fail(ctx, ABP_EINVAL, "set %d: L = %g must be > 0", i, p.L);
        if (p.D < 0.0) return fail(ctx, ABP_EINVAL, "set %d: D = %g must be >= 0", i, p.D);
        if (n_traj[i] < 0) return fail(ctx, ABP_EINVAL, "set %d: n_traj < 0", i);
        if (n_steps[i] < 0 || n_steps[i] >= kMaxSteps)
            return fail(ctx, ABP_EINVAL, "set %d: n_steps = %lld outside [0, 2^34)", i, (long long)n_steps[i]);
        total += n_traj[i];
        if (total > ((int64_t)1 << 40)) return fail(ctx, ABP_EINVAL, "too many trajectories");
        max_n = std::max(max_n, n_steps[i]);
    }
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    if (se != cudaSuccess) return cuda_fail(ctx, se, "synchronise before new batch");
    ctx->release_batch();

    ctx->n_sets = n_sets;
    ctx->params.assign(sets, sets + n_sets);
    ctx->n_traj.assign(n_traj, n_traj + n_sets);
    ctx->n_steps.assign(n_steps, n_steps + n_sets);
    ctx->total_traj = total;
    ctx->max_steps = max_n;
    ctx->g = 0;

    // Tiles: contiguous runs of at most kThreads * ppt trajectories of one set.
    const int64_t tile = (int64_t)kThreads * ctx->ppt;
    ctx->set_tile_begin.assign(1, 0);
    ctx->tile_first.clear();
    ctx->tile_count.clear();
    ctx->tile_set.clear();
    int64_t base = 0;
    for (int32_t i = 0; i < n_sets; ++i) {
        for (int64_t off = 0; off < n_traj[i]; off += tile) {
            ctx->tile_first.push_back(base + off);
            ctx->tile_count.push_back((int32_t)std::min(tile, n_traj[i] - off));
            ctx->tile_set.push_back(i);
        }
        if (ctx->tile_first.size() > (size_t)INT32_MAX - 1) return fail(ctx, ABP_EINVAL, "too many tiles");
        ctx->set_tile_begin.push_back((int32_t)ctx->tile_first.size());
        base += n_traj[i];
    }
    ctx->n_tiles = (int32_t)ctx->tile_first.size();
    const abp_config &c = ctx->cfg;
    const bool any_hist = c.hist_x_bins > 0 || c.hist_v_bins > 0;
    ctx->n_snap = any_hist ? (c.snapshot_every > 0 ? max_n / c.snapshot_every : 1) : 0;
    ctx->n_ckpt = c.checkpoint_every > 0 ? max_n / c.checkpoint_every + 1 : 0;
    ctx->steps_per_launch = c.steps_per_launch > 0 ? c.steps_per_launch : default_steps_per_launch(ctx);

    const size_t T = (size_t)total;
    const size_t rsz = c.state_fp64 ? sizeof(double) : sizeof(float);
    abp_status st = ABP_OK;
#define ALLOC(buf, bytes, what) \
    if ((st = alloc(ctx, ctx->buf, (bytes), what)) != ABP_OK) { ctx->release_all(); return st; }
    ALLOC(d_params, sizeof(abp_params) * (size_t)n_sets, "parameters");
    ALLOC(d_steps, sizeof(int64_t) * (size_t)n_sets, "step counts");
    ALLOC(d_set_tile_begin, sizeof(int32_t) * ((size_t)n_sets + 1), "set tiles");
    ALLOC(d_tile_first, sizeof(int64_t) * (size_t)ctx->n_tiles, "tile table");
    ALLOC(d_tile_count, sizeof(int32_t) * (size_t)ctx->n_tiles, "tile table");
    ALLOC(d_tile_set, sizeof(int32_t) * (size_t)ctx->n_tiles, "tile table");
    ALLOC(d_y, rsz * T, "state y");
    ALLOC(d_yacc, rsz * T, "state yacc");
    ALLOC(d_ylo, rsz * T, "state ylo");
    ALLOC(d_v, rsz * T, "state v");
    ALLOC(d_e, rsz * T, "state e");
    ALLOC(d_y0, rsz * T, "state y0");
    ALLOC(d_cell, sizeof(int32_t) * T, "state cell");
    ALLOC(d_hx, sizeof(uint32_t) * (size_t)ctx->n_snap * n_sets * (size_t)std::max(c.hist_x_bins, 0), "x histograms");
    ALLOC(d_hv, sizeof(uint32_t) * (size_t)ctx->n_snap * n_sets * (size_t)(c.hist_v_bins > 0 ? c.hist_v_bins + 2 : 0),
          "v histograms");
    ALLOC(d_ckpt, sizeof(float4) * (size_t)ctx->n_ckpt * T, "checkpoints");
    ALLOC(d_partials, sizeof(double) * 4 * (size_t)std::max(ctx->n_tiles, 1), "reduction scratch");
    ALLOC(d_moments, sizeof(double) * 8 * (size_t)std::max(n_sets, 1), "moments");
#undef ALLOC

    cudaStream_t s = ctx->stream;
    auto up = [&](DevBuf &b, const void *src, size_t n) -> cudaError_t {
        return n ? cudaMemcpyAsync(b.p, src, n, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    cudaError_t e = up(ctx->d_params, ctx->params.data(), sizeof(abp_params) * n_sets);
    if (e == cudaSuccess) e = up(ctx->d_steps, ctx->n_steps.data(), sizeof(int64_t) * n_sets);
    if (e == cudaSuccess) e = up(ctx->d_set_tile_begin, ctx->set_tile_begin.data(), sizeof(int32_t) * (n_sets + 1));
    if (e == cudaSuccess) e = up(ctx->d_tile_first, ctx->tile_first.data(), sizeof(int64_t) * ctx->n_tiles);
    if (e == cudaSuccess) e = up(ctx->d_tile_count, ctx->tile_count.data(), sizeof(int32_t) * ctx->n_tiles);
    if (e == cudaSuccess) e = up(ctx->d_tile_set, ctx->tile_set.data(), sizeof(int32_t) * ctx->n_tiles);
    if (e == cudaSuccess && ctx->d_hx.bytes) e = cudaMemsetAsync(ctx->d_hx.p, 0, ctx->d_hx.bytes, s);
    if (e == cudaSuccess && ctx->d_hv.bytes) e = cudaMemsetAsync(ctx->d_hv.p, 0, ctx->d_hv.bytes, s);
    if (e == cudaSuccess) {
        e = launch_init(ctx->batch(), ctx->state(), ctx->hist(), ctx->ckpt(), ctx->noise(), s);
        ctx->launches += ctx->n_tiles > 0 ? 1 : 0;
    }
    // The host arrays above are pageable vectors owned by the context; make the
    // uploads complete before the context can be modified again.
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ctx->release_batch();
        return cuda_fail(ctx, e, "upload / initial condition");
    }
    ctx->have_batch = true;
    return ABP_OK;
}

abp_status abp_reset(abp_ctx *ctx, uint64_t seed) {
    if (!ctx) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_reset before abp_set_params");
    ctx->cfg.seed = seed;
    ctx->g = 0;
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaSuccess;
    if (ctx->d_hx.bytes) e = cudaMemsetAsync(ctx->d_hx.p, 0, ctx->d_hx.bytes, s);
    if (e == cudaSuccess && ctx->d_hv.bytes) e = cudaMemsetAsync(ctx->d_hv.p, 0, ctx->d_hv.bytes, s);
    if (e == cudaSuccess) {
        e = launch_init(ctx->batch(), ctx->state(), ctx->hist(), ctx->ckpt(), ctx->noise(), s);
        ctx->launches += ctx->n_tiles > 0 ? 1 : 0;
    }
    return e == cudaSuccess ? ABP_OK : cuda_fail(ctx, e, "reset");
}

abp_status abp_kernel_launches(const abp_ctx *ctx, int64_t *launches) {
    if (!ctx || !launches) return ABP_EINVAL;
    *launches = ctx->launches;
    return ABP_OK;
}

abp_status abp_integrate(abp_ctx *ctx, int64_t max_steps) {
    if (!ctx) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_integrate before abp_set_params");
    const int64_t target = max_steps < 0 ? ctx->max_steps : std::min(ctx->max_steps, ctx->g + max_steps);
    const Batch b = ctx->batch();
    const State s = ctx->state();
    const Hist h = ctx->hist();
    const Ckpt c = ctx->ckpt();
    const Noise nz = ctx->noise();
    while (ctx->g < target) {
        const int64_t g1 = std::min(target, ctx->g + ctx->steps_per_launch);
        cudaError_t e = launch_integrate(b, s, h, c, nz, ctx->ppt, ctx->g, g1, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "integrator launch");
        ctx->launches += b.n_tiles > 0 ? 1 : 0;
        ctx->g = g1;
    }
    return ABP_OK;
}

abp_status abp_progress(const abp_ctx *ctx, int64_t *steps_done) {
    if (!ctx || !steps_done) return ABP_EINVAL;
    for (int32_t i = 0; i < ctx->n_sets; ++i) steps_done[i] = std::min(ctx->g, ctx->n_steps[i]);
    return ABP_OK;
}

abp_status abp_num_snapshots(const abp_ctx *ctx, int64_t *n_snap) {
    if (!ctx || !n_snap) return ABP_EINVAL;
    *n_snap = ctx->n_snap;
    return ABP_OK;
}

abp_status abp_reduce(abp_ctx *ctx, double *moments, uint32_t *hist_x, uint32_t *hist_v) {
    if (!ctx) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_reduce before abp_set_params");
    bool synced = false;
    abp_status st;
    if (moments) {
        cudaError_t e = launch_reduce(ctx->batch(), ctx->state(), ctx->noise(), ctx->g, (double *)ctx->d_partials.p,
                                      (double *)ctx->d_moments.p, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "reduction launch");
        ctx->launches += (ctx->n_tiles > 0 ? 1 : 0) + (ctx->n_sets > 0 ? 1 : 0);
        if ((st = deliver(ctx, moments, ctx->d_moments.p, sizeof(double) * 8 * ctx->n_sets, &synced)) != ABP_OK)
            return st;
    }
    if (hist_x && ctx->d_hx.bytes)
        if ((st = deliver(ctx, hist_x, ctx->d_hx.p, ctx->d_hx.bytes, &synced)) != ABP_OK) return st;
    if (hist_v && ctx->d_hv.bytes)
        if ((st = deliver(ctx, hist_v, ctx->d_hv.p, ctx->d_hv.bytes, &synced)) != ABP_OK) return st;
    if (synced) return abp_synchronize(ctx);
    return ABP_OK;
}

abp_status abp_get_state(abp_ctx *ctx, double *x, double *x0, double *v, double *e, double *vbar) {
    if (!ctx) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_get_state before abp_set_params");
    double *outs[5] = {x, x0, v, e, vbar};
    const size_t n = (size_t)ctx->total_traj;
    bool all_dev = true;
    for (double *p : outs)
        if (p && !is_device_ptr(p)) all_dev = false;
    if (all_dev) {
        cudaError_t er = launch_get_state(ctx->batch(), ctx->state(), ctx->cfg.dt, ctx->g, x, x0, v, e, vbar, ctx->stream);
        ctx->launches += ctx->n_tiles > 0 ? 1 : 0;
        return er == cudaSuccess ? ABP_OK : cuda_fail(ctx, er, "state readback");
    }
    DevBuf tmp;
    abp_status st = alloc(ctx, tmp, sizeof(double) * 5 * std::max<size_t>(n, 1), "state readback");
    if (st != ABP_OK) return st;
    double *t = (double *)tmp.p;
    double *d[5];
    for (int i = 0; i < 5; ++i) d[i] = outs[i] ? t + i * n : nullptr;
    cudaError_t er = launch_get_state(ctx->batch(), ctx->state(), ctx->cfg.dt, ctx->g, d[0], d[1], d[2], d[3], d[4], ctx->stream);
    ctx->launches += ctx->n_tiles > 0 ? 1 : 0;
    bool synced = false;
    for (int i = 0; i < 5 && er == cudaSuccess; ++i)
        if (outs[i]) {
            st = deliver(ctx, outs[i], d[i], sizeof(double) * n, &synced);
            if (st != ABP_OK) break;
        }
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    tmp.release();
    if (er != cudaSuccess) return cuda_fail(ctx, er, "state readback");
    if (st != ABP_OK) return st;
    if (se != cudaSuccess) return cuda_fail(ctx, se, "state readback");
    return ABP_OK;
}

abp_status abp_synchronize(abp_ctx *ctx) {
    if (!ctx) return ABP_EINVAL;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronise");
    int32_t status = 0;
    e = cudaMemcpy(&status, ctx->d_status.p, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status readback");
    if (status == 1) return fail(ctx, ABP_ETIMEOUT, "a bounded device-side wait expired");
    if (status != 0) return fail(ctx, ABP_ESTATE, "device reported status %d", status);
    return ABP_OK;
}

abp_status abp_backward(abp_ctx *ctx, const double *dJ_dmean_v, double *grad);  // abp_adjoint.cu

abp_status abp_philox(uint64_t seed, const uint64_t *traj, const uint64_t *m, int64_t n, uint32_t *out,
                      void *cuda_stream) {
    if (n < 0) return ABP_EINVAL;
    if (n == 0) return ABP_OK;
    if (!traj || !m || !out || !is_device_ptr(traj) || !is_device_ptr(m) || !is_device_ptr(out)) return ABP_EINVAL;
    cudaError_t e = launch_philox((uint32_t)seed, (uint32_t)(seed >> 32), traj, m, n, out, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? ABP_OK : ABP_ECUDA;
}

abp_status abp_normals(uint64_t seed, uint64_t traj, uint64_t n0, int64_t count, float *out, void *cuda_stream) {
    if (count < 0) return ABP_EINVAL;
    if (count == 0) return ABP_OK;
    if (!out || !is_device_ptr(out)) return ABP_EINVAL;
    cudaError_t e = launch_normals((uint32_t)seed, (uint32_t)(seed >> 32), traj, n0, count, out,
                                   (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? ABP_OK : ABP_ECUDA;
}

}  // extern "C"
