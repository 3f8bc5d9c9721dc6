// abp_api.cu -- host runtime of the C ABI declared in include/abp.h.
//
// Owns the device buffers of a batch (structure-of-arrays trajectory state,
// tile table, histograms, adjoint checkpoints, reduction scratch), validates
// every argument, tiles the parameter sets for the device and enqueues the
// kernels of abp_kernels.cu / abp_adjoint.cu on the context's stream.
#include <dlfcn.h>
#include <unistd.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
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
// Resident blocks per SM of the work queue for a batch of n_tiles tiles: the
// kernel's occupancy, but no more blocks than leave 1.5 tiles to each.  An item
// waits for its tile's previous round; with about one tile per block the blocks
// of a round outrun the tiles and idle on those waits (load sweep, 512 tiles:
// 9.95e11 particle-steps/s on 304 blocks, 9.64e11 on 456).  One block already
// draws an SM's full rate, so fewer blocks cost little elsewhere.
int wq_blocks_per_sm(int bps, int64_t n_tiles, int sms) {
    const int64_t fit = (2 * n_tiles) / (3 * (int64_t)std::max(sms, 1));
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::max(bps, 1), fit));
}

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

bool finite_params(const abp_params &p) {
    const double v[9] = {p.q, p.c, p.d, p.gamma0, p.F0, p.D, p.h, p.L, p.asym};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

// Equal windows of about 2e10 particle-steps each (tens of ms on a GB300),
// a multiple of 64 steps.
int64_t default_window(int64_t total_traj, int64_t max_steps) {
    if (total_traj == 0 || max_steps == 0) return std::max<int64_t>(max_steps, 1);
    const double work = (double)total_traj * (double)max_steps;
    const int64_t n_launch = std::max<int64_t>(1, (int64_t)std::ceil(work / 2.0e10));
    int64_t s = (max_steps + n_launch - 1) / n_launch;
    s = ((s + 63) / 64) * 64;
    return std::max<int64_t>(1, std::min<int64_t>(s, max_steps));
}

// Copy n bytes of a device buffer to a caller pointer that may be host or device.
abp_status deliver(abp_ctx *ctx, void *dst, const void *src, size_t n, bool *synced) {
    if (!dst || n == 0) return ABP_OK;
    const PtrKind k = ptr_kind(dst, ctx->device);
    if (k == PtrKind::OtherDevice)
        return fail(ctx, ABP_EINVAL, "an output points to another GPU's memory (the context runs on device %d)",
                    ctx->device);
    if (k == PtrKind::Device) {
        ABP_CUDA(ctx, cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, ctx->stream), "copy to device output");
    } else {
        ABP_CUDA(ctx, cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, ctx->stream), "copy to host output");
        *synced = true;
    }
    return ABP_OK;
}

// ---------------------------------------------------------------- autotuner

// Schedule and particles per thread.  Every (schedule, PPT) candidate is timed
// once per device and state type on a synthetic single-set batch several
// waves deep (4,096 trajectories per SM, 8,192 steps after a 256-step warm-up,
// CUDA events on the context's stream); choose_configuration() weighs the
// table with the batch at hand.
struct TuneTable {
    bool done = false;
    float ms[3][3] = {};  // [schedule 1 = lockstep, 2 = work queue][ppt 1, 2, 4]
};
TuneTable g_tune[64][4];

// Kind of integrator a timing table belongs to: 0 FP32 Euler-Maruyama, 1 FP64
// state, 2 FP32 stochastic Heun, 3 FP32 Euler-Maruyama with xorshift noise.
int tune_kind(const abp_ctx *ctx) {
    return ctx->cfg.state_fp64 ? 1 : ctx->cfg.scheme == 1 ? 2 : ctx->cfg.noise == 1 ? 3 : 0;
}

// The autotuner's trial batch: one set of kTrialTrajPerSm trajectories per SM,
// kTrialSteps timed steps, run by the work queue as kTrialRounds rounds (as
// real batches run it).
constexpr int64_t kTrialTrajPerSm = 4096;
constexpr int64_t kTrialSteps = 8192;
constexpr int kTrialRounds = 4;

void measure_candidates(abp_ctx *ctx, TuneTable &tt) {
    const int fp = ctx->cfg.state_fp64 ? 1 : 0;
    const bool heun = ctx->cfg.scheme == 1;
    const int64_t T = (int64_t)std::max(ctx->sm_count, 1) * kTrialTrajPerSm;
    const int64_t warm = 256, steps = kTrialSteps;
    const size_t rsz = fp ? sizeof(double) : sizeof(float);
    const int cands[3] = {1, 2, 4};
    const int max_tiles = (int)((T + kThreads - 1) / kThreads);
    const bool xorshift = ctx->cfg.noise == 1;
    const size_t bytes =
        256 * 16 + (sizeof(int64_t) + 5 * sizeof(int32_t)) * max_tiles + (6 * rsz + 4 + (xorshift ? 16 : 0)) * T + 8192;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) tt.ms[i][j] = 1e30f;
    void *mem = nullptr;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    char *p = (char *)mem;
    auto take = [&](size_t n) {
        char *r = p;
        p += (n + 255) & ~(size_t)255;
        return r;
    };
    abp_params prm{1.0, 0.1, 1.0, 1.0, 0.0, 0.1, 1.0, 1.0, 0.25};
    const int64_t nsteps = warm + steps;
    abp_params *d_prm = (abp_params *)take(sizeof(abp_params));
    int64_t *d_steps = (int64_t *)take(sizeof(int64_t));
    int32_t *d_stb = (int32_t *)take(2 * sizeof(int32_t));
    int64_t *d_first = (int64_t *)take(sizeof(int64_t) * max_tiles);
    int32_t *d_count = (int32_t *)take(sizeof(int32_t) * max_tiles);
    int32_t *d_tset = (int32_t *)take(sizeof(int32_t) * max_tiles);
    State st;
    st.fp64 = fp != 0;
    st.y = take(rsz * T);
    st.yacc = take(rsz * T);
    st.ylo = take(rsz * T);
    st.v = take(rsz * T);
    st.e = take(rsz * T);
    st.y0 = take(rsz * T);
    st.cell = (int32_t *)take(sizeof(int32_t) * T);
    st.xs = xorshift ? (uint4 *)take(sizeof(uint4) * T) : nullptr;
    int32_t *d_queue = (int32_t *)take(sizeof(int32_t) * ((size_t)max_tiles + 1));
    int32_t *d_perm = (int32_t *)take(sizeof(int32_t) * max_tiles);
    int32_t *d_rs = (int32_t *)take(sizeof(int32_t) * (kTrialRounds + 1));
    int32_t *d_status = (int32_t *)take(sizeof(int32_t));
    Hist h{};
    Ckpt ck{};
    Noise nz{};
    nz.dt = 1e-3;
    nz.scheme = heun ? 1 : 0;
    nz.noise = xorshift ? 1 : 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaStream_t s = ctx->stream;
    for (int ci = 0; ci < 3; ++ci) {
        const int c = cands[ci];
        const int64_t tile = (int64_t)kThreads * c;
        const int nt = (int)((T + tile - 1) / tile);
        std::vector<int64_t> first(nt);
        std::vector<int32_t> count(nt), tset(nt, 0), perm(nt);
        for (int t = 0; t < nt; ++t) {
            first[t] = t * tile;
            count[t] = (int32_t)std::min<int64_t>(tile, T - t * tile);
            perm[t] = t;
        }
        const int32_t stb[2] = {0, nt};
        int32_t rs[kTrialRounds + 1];
        for (int r = 0; r <= kTrialRounds; ++r) rs[r] = r * nt;
        cudaMemcpyAsync(d_prm, &prm, sizeof(prm), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_steps, &nsteps, sizeof(nsteps), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_stb, stb, sizeof(stb), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_first, first.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_count, count.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_tset, tset.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_perm, perm.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_rs, rs, sizeof(rs), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(d_status, 0, sizeof(int32_t), s);
        Batch b;
        b.n_sets = 1;
        b.n_tiles = nt;
        b.n_single = nt;
        b.set_first = nullptr;
        b.set_order = nullptr;
        b.slot_set = nullptr;
        b.n_unpacked = 1;
        b.narrow = 0;
        b.sub_single = b.sub_packed = 1;
        b.total_traj = T;
        b.params = d_prm;
        b.set_steps = d_steps;
        b.set_tile_begin = d_stb;
        b.tile_first = d_first;
        b.tile_count = d_count;
        b.tile_set = d_tset;
        int bps = 0;
        persistent_occupancy(fp != 0, c, 0, &bps, heun ? 1 : xorshift ? 2 : 0);
        Queue q;
        q.head = d_queue;
        q.done = d_queue + 1;
        q.status = d_status;
        q.round_start = d_rs;
        q.perm = d_perm;
        q.n_rounds = 1;
        q.n_items = nt;
        q.hold_tile = -1;
        q.wait_limit_ns = 10000000000LL;
        const int grid = std::min(wq_blocks_per_sm(bps, nt, ctx->sm_count) * std::max(ctx->sm_count, 1), nt);
        for (int sch = 1; sch <= 2; ++sch) {
            auto window = [&](int64_t g0, int64_t g1) {
                if (sch == 1) {
                    launch_integrate(b, st, h, ck, nz, c, g0, g1, s);
                } else {
                    cudaMemsetAsync(d_queue, 0, sizeof(int32_t) * ((size_t)nt + 1), s);
                    // the warm-up as one round, the timed window as kTrialRounds rounds
                    Queue qw = q;
                    const int rounds = g0 == 0 ? 1 : kTrialRounds;
                    qw.n_rounds = rounds;
                    qw.n_items = rounds * nt;
                    launch_persistent(b, st, h, ck, nz, qw, c, grid, g0, g1, (g1 - g0) / rounds, s);
                }
            };
            launch_init(b, st, h, ck, nz, s);
            window(0, warm);
            cudaEventRecord(e0, s);
            window(warm, warm + steps);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f) tt.ms[sch][ci] = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(mem);
    cudaGetLastError();
    tt.done = true;
}

// The timing table is also kept on disk beside the library (one line per
// device model, SM count, state type and library build), so that every
// process on the machine -- including a profiled rerun, whose own timings
// would be distorted by the profiler -- makes the same choice.
std::string tune_cache_path() {
    // ABP_TUNE_FILE relocates the file (a read-only installation, or one file shared by
    // several builds' users); an empty value switches the file off
    if (const char *env = getenv("ABP_TUNE_FILE")) return std::string(env);
    Dl_info info;
    if (!dladdr((const void *)&abp_version, &info) || !info.dli_fname) return std::string();
    std::string p(info.dli_fname);
    const size_t slash = p.rfind('/');
    return (slash == std::string::npos ? std::string(".") : p.substr(0, slash)) + "/abp_tune_cache.txt";
}

std::string tune_key(const abp_ctx *ctx) {
    cudaDeviceProp prop;
    char name[256] = "unknown";
    if (cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess) snprintf(name, sizeof(name), "%s", prop.name);
    cudaGetLastError();
    for (char *c = name; *c; ++c)
        if (*c == ' ' || *c == '|') *c = '_';
    char key[512];
    // the build time stamp: every rebuild of the library re-times the candidates
    snprintf(key, sizeof(key), "%s|%d|%d|%s|%s_%s", name, ctx->sm_count, tune_kind(ctx), abp_version(), __DATE__,
             __TIME__);
    for (char *c = key; *c; ++c)
        if (*c == ' ') *c = '_';
    return key;
}

bool load_tune(const abp_ctx *ctx, TuneTable &tt) {
    const std::string path = tune_cache_path(), key = tune_key(ctx);
    if (path.empty()) return false;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    char line[1024];
    bool ok = false;
    while (fgets(line, sizeof(line), f)) {
        char k[512];
        float m[6];
        if (sscanf(line, "%511s %f %f %f %f %f %f", k, &m[0], &m[1], &m[2], &m[3], &m[4], &m[5]) == 7 && key == k) {
            for (int i = 0; i < 3; ++i) {
                tt.ms[1][i] = m[i];
                tt.ms[2][i] = m[3 + i];
            }
            tt.done = ok = true;
        }
    }
    fclose(f);
    return ok;
}

void save_tune(const abp_ctx *ctx, const TuneTable &tt) {
    const std::string path = tune_cache_path(), key = tune_key(ctx);
    if (path.empty()) return;
    std::vector<std::string> keep;
    if (FILE *f = fopen(path.c_str(), "r")) {
        char line[1024];
        while (fgets(line, sizeof(line), f)) {
            char k[512];
            if (sscanf(line, "%511s", k) == 1 && key != k) keep.emplace_back(line);
        }
        fclose(f);
    }
    const std::string tmp = path + ".tmp." + std::to_string((long)getpid());
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const std::string &l : keep) fputs(l.c_str(), f);
    fprintf(f, "%s %.6g %.6g %.6g %.6g %.6g %.6g\n", key.c_str(), tt.ms[1][0], tt.ms[1][1], tt.ms[1][2], tt.ms[2][0],
            tt.ms[2][1], tt.ms[2][2]);
    fclose(f);
    if (rename(tmp.c_str(), path.c_str()) != 0) remove(tmp.c_str());
}

// Choices of the probe are kept in the same file, one line "C|<table key>|<batch key>
// schedule ppt steps" each, so that a rerun of the same program (a profiled one, whose
// probe timings would be distorted) runs the same configuration.
bool load_choice(const abp_ctx *ctx, uint64_t bkey, int *sched, int *ppt, int64_t *spl) {
    const std::string path = tune_cache_path();
    if (path.empty()) return false;
    char want[640];
    snprintf(want, sizeof(want), "C|%s|%016llx", tune_key(ctx).c_str(), (unsigned long long)bkey);
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    char line[1024];
    bool ok = false;
    while (fgets(line, sizeof(line), f)) {
        char k[640];
        int a = 0, b = 0;
        long long c = 0;
        if (sscanf(line, "%639s %d %d %lld", k, &a, &b, &c) == 4 && strcmp(k, want) == 0 && (a == 1 || a == 2) &&
            (b == 1 || b == 2 || b == 4) && c > 0) {
            *sched = a;
            *ppt = b;
            *spl = c;
            ok = true;
        }
    }
    fclose(f);
    return ok;
}

void save_choice(const abp_ctx *ctx, uint64_t bkey, int sched, int ppt, int64_t spl) {
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    char want[640];
    snprintf(want, sizeof(want), "C|%s|%016llx", tune_key(ctx).c_str(), (unsigned long long)bkey);
    std::vector<std::string> keep;
    if (FILE *f = fopen(path.c_str(), "r")) {
        char line[1024];
        while (fgets(line, sizeof(line), f)) {
            char k[640];
            if (sscanf(line, "%639s", k) == 1 && strcmp(k, want) != 0) keep.emplace_back(line);
        }
        fclose(f);
    }
    const std::string tmp = path + ".tmp." + std::to_string((long)getpid());
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const std::string &l : keep) fputs(l.c_str(), f);
    fprintf(f, "%s %d %d %lld\n", want, sched, ppt, (long long)spl);
    fclose(f);
    if (rename(tmp.c_str(), path.c_str()) != 0) remove(tmp.c_str());
}

// Fraction of a candidate's launch capacity that the batch keeps busy, in
// particle-steps: lockstep runs the tiles that still have steps in each window
// of the default length, in waves of `cap` resident blocks (small sets of
// equal step count share packed tiles); the work queue balances all
// tile-steps over `cap` blocks, plus half a work item of tail, bounded below by
// the longest tile's chain.
// A tile of kThreads * ppt slots costs the same however full it is.
// The fraction of `units` parallel units a batch keeps busy, in particle-steps.
// The autotuner passes the SM count: one resident block already draws its SM's
// full integration rate (measured: time against tiles per SM is a staircase in
// ceil(tiles / SMs) for both schedules, with one, two or three blocks per SM), so
// a batch's last partial round costs whole tiles per SM, not per block.
double batch_efficiency(int32_t n, const int64_t *n_traj, const int64_t *n_steps, int sched, int ppt,
                        bool checkpoints, int64_t spl, int64_t units) {
    const int64_t cap = units;
    const int64_t slots = (int64_t)kThreads * ppt;
    std::vector<std::pair<int64_t, int64_t>> tiles;  // (tile count, steps)
    std::map<int64_t, int64_t> small;               // steps -> trajectories of small sets (lockstep packs them)
    double useful = 0.0;
    int64_t max_n = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int64_t M = n_traj[i], N = n_steps[i];
        if (M <= 0 || N <= 0) continue;
        useful += (double)M * (double)N;
        max_n = std::max(max_n, N);
        if (sched == 1 && !checkpoints && M < kThreads)
            small[N] += M;
        else
            tiles.emplace_back((M + slots - 1) / slots, N);
    }
    for (const auto &kv : small) tiles.emplace_back((kv.second + kThreads - 1) / kThreads, kv.first);
    if (useful <= 0.0 || cap <= 0) return 1.0;
    double cost = 0.0;  // particle-step capacity spent
    if (sched == 2) {
        // list scheduling of the work items on the units: when every tile has the same
        // step count and the items divide it, all items are equal and the makespan is
        // ceil(items / units) items; otherwise about W / units plus half an item.  Never
        // less than the longest tile, whose items run one after another.  Items of spl
        // steps (0: the largest of 10^5, 10^4, 10^3 giving 32 items per unit).
        double tile_steps = 0.0;
        bool equal = true;
        for (const auto &t : tiles) {
            tile_steps += (double)t.first * (double)t.second;
            equal = equal && t.second == tiles[0].second;
        }
        int64_t item = spl > 0 ? spl : 1000;
        for (int64_t S : {100000, 10000, 1000}) {
            if (spl > 0) break;
            int64_t items = 0;
            for (const auto &t : tiles) items += t.first * ((t.second + S - 1) / S);
            if (items >= 32 * cap) {
                item = S;
                break;
            }
        }
        double span;
        if (equal && (max_n <= item || max_n % item == 0)) {
            const int64_t len = std::min(item, max_n);
            int64_t items = 0;
            for (const auto &t : tiles) items += t.first * (max_n / len);
            span = (double)((items + cap - 1) / cap) * (double)len;
        } else {
            span = tile_steps / (double)cap + 0.5 * (double)std::min(item, max_n);
        }
        span = std::max(span, (double)max_n);
        cost = (double)cap * span * (double)slots;
    } else {
        spl = std::max<int64_t>(spl, 1);
        for (int64_t g = 0; g < max_n; g += spl) {
            int64_t active = 0, len = 0;
            for (const auto &t : tiles)
                if (t.second > g) {
                    active += t.first;
                    len = std::max(len, std::min(t.second, g + spl) - g);
                }
            cost += (double)((active + cap - 1) / cap) * (double)cap * (double)len * (double)slots;
        }
    }
    return cost > 0.0 ? std::min(1.0, useful / cost) : 1.0;
}

// The tiling of a batch (host only).  Tiles are contiguous runs of at most
// kThreads * ppt trajectories of one set, followed -- lockstep schedule, no
// adjoint checkpoints -- by packed tiles: runs of consecutive small sets (fewer
// than kThreads trajectories each, equal step counts, at least two non-empty)
// sharing one block, one trajectory per thread.  A lockstep batch with fewer
// tiles than SMs is launched narrow: blocks of the widest w in {256, 128, 64}
// that still gives every SM a block (else 32), one trajectory per thread.
struct TilePlan {
    std::vector<int64_t> set_first, tile_first;
    std::vector<int32_t> set_packed, set_tile_begin, tile_count, tile_set, set_order;
    std::vector<int32_t> slot_set;  // [packed tiles][kThreads]: the set of each slot's trajectory
    int32_t n_single = 0, n_unpacked = 0, narrow = 0, sub_single = 1, sub_packed = 1;
};

bool plan_tiles(int32_t n_sets, const int64_t *n_traj, const int64_t *n_steps, int sched, int ppt, bool checkpoints,
                int sm_count, TilePlan &p) {
    const int64_t tile = (int64_t)kThreads * ppt;
    const bool can_pack = sched == 1 && !checkpoints;
    p.set_first.assign((size_t)n_sets + 1, 0);
    for (int32_t i = 0; i < n_sets; ++i) p.set_first[i + 1] = p.set_first[i] + n_traj[i];
    p.set_packed.assign((size_t)n_sets, 0);
    std::vector<std::pair<int32_t, int32_t>> groups;  // [first set, end set) of each packed tile
    if (can_pack) {
        int32_t i = 0;
        while (i < n_sets) {
            if (n_traj[i] <= 0 || n_traj[i] >= kThreads) {
                ++i;
                continue;
            }
            int32_t j = i, nonempty = 0;
            int64_t cnt = 0;
            while (j < n_sets && (n_traj[j] == 0 || (n_traj[j] < kThreads && n_steps[j] == n_steps[i])) &&
                   cnt + n_traj[j] <= kThreads) {
                cnt += n_traj[j];
                nonempty += n_traj[j] > 0 ? 1 : 0;
                ++j;
            }
            if (nonempty >= 2) {
                groups.emplace_back(i, j);
                for (int32_t k = i; k < j; ++k) p.set_packed[k] = n_traj[k] > 0 ? 1 : 0;
            }
            i = j > i ? j : i + 1;
        }
    }
    p.set_tile_begin.assign(1, 0);
    p.tile_first.clear();
    p.tile_count.clear();
    p.tile_set.clear();
    for (int32_t i = 0; i < n_sets; ++i) {
        if (!p.set_packed[i])
            for (int64_t off = 0; off < n_traj[i]; off += tile) {
                p.tile_first.push_back(p.set_first[i] + off);
                p.tile_count.push_back((int32_t)std::min(tile, n_traj[i] - off));
                p.tile_set.push_back(i);
            }
        if (p.tile_first.size() > (size_t)INT32_MAX / 2) return false;
        p.set_tile_begin.push_back((int32_t)p.tile_first.size());
    }
    p.n_single = (int32_t)p.tile_first.size();
    p.slot_set.clear();
    for (const auto &gr : groups) {
        int32_t lead = gr.first;
        while (n_traj[lead] == 0) ++lead;  // the first non-empty set carries the group's step count
        p.tile_first.push_back(p.set_first[gr.first]);
        p.tile_count.push_back((int32_t)(p.set_first[gr.second] - p.set_first[gr.first]));
        p.tile_set.push_back(lead);
        // slot li holds trajectory tile_first + li (slots past the count repeat the last set)
        int32_t k = lead;
        for (int64_t li = 0; li < kThreads; ++li) {
            const int64_t t = p.set_first[gr.first] + std::min<int64_t>(li, p.tile_count.back() - 1);
            while (k + 1 < gr.second && p.set_first[k + 1] <= t) ++k;
            p.slot_set.push_back(k);
        }
    }
    const int32_t n_tiles = (int32_t)p.tile_first.size();
    p.set_order.clear();
    for (int32_t i = 0; i < n_sets; ++i)
        if (!p.set_packed[i]) p.set_order.push_back(i);
    p.n_unpacked = (int32_t)p.set_order.size();
    for (int32_t i = 0; i < n_sets; ++i)
        if (p.set_packed[i]) p.set_order.push_back(i);
    p.narrow = 0;
    p.sub_single = p.sub_packed = 1;
    if (sched == 1 && n_tiles > 0 && n_tiles < sm_count) {
        int w = 32;
        for (int cand : {256, 128, 64}) {
            if (cand >= tile) continue;
            int64_t blocks = 0;
            for (int32_t t = 0; t < n_tiles; ++t) blocks += (p.tile_count[t] + cand - 1) / cand;
            if (blocks >= sm_count) {
                w = cand;
                break;
            }
        }
        p.narrow = w;
        p.sub_single = (int32_t)((tile + w - 1) / w);
        p.sub_packed = kThreads / w;
    }
    return true;
}

// The autotuner's model of a candidate (schedule, trajectories per thread, steps per
// launch) on a batch: the candidate's trial time brought to full use of the SMs, scaled
// to the batch's particle-steps and divided by the fraction of the SMs the batch keeps
// busy (batch_efficiency), plus what its launches move and cost -- every lockstep
// window loads and stores the state of the trajectories still running, every work item
// that of its tile (at the device copy rate), and each launch or item pop has a fixed cost.
// The constants are measured on GB300: copy rate ~6.7 TB/s, a graph-replayed launch a few
// microseconds, one item's pop, wait and publish about two microseconds of a block.
constexpr double kHbmBytesPerMs = 6.5e9;
// Candidates within this fraction of their schedule's best model time are probed too.
constexpr double kProbeBand = 0.03;
constexpr double kLaunchMs = 0.03;
constexpr double kItemMs = 0.002;

// Bytes of trajectory state a launch reads and writes per trajectory.
double state_io_bytes(const abp_config &c) {
    return 2.0 * ((c.state_fp64 ? 8.0 : 4.0) * 6.0 + 4.0 + (c.noise == 1 ? 16.0 : 0.0));
}

// Blocks of a candidate's integrator resident at once.
int64_t candidate_capacity(const abp_ctx *ctx, int sched, int ppt) {
    const abp_config &c = ctx->cfg;
    const size_t smem = sizeof(uint32_t) * (size_t)(c.hist_x_bins + (c.hist_v_bins > 0 ? c.hist_v_bins + 2 : 0));
    const int mode = c.scheme == 1 ? 1 : c.noise == 1 ? 2 : 0;
    int bps = 0;
    const cudaError_t oe = sched == 1 ? integrate_occupancy(c.state_fp64 != 0, ppt, smem, &bps, mode)
                                      : persistent_occupancy(c.state_fp64 != 0, ppt, smem, &bps, mode);
    if (oe != cudaSuccess) cudaGetLastError();
    if (sched == 2) {
        int64_t tiles = 0;
        for (int32_t i = 0; i < ctx->n_sets; ++i) tiles += (ctx->n_traj[i] + kThreads * ppt - 1) / (kThreads * ppt);
        bps = wq_blocks_per_sm(bps, tiles, ctx->sm_count);
    }
    return (int64_t)std::max(bps, 1) * std::max(ctx->sm_count, 1);
}

int ppt_index(int ppt) { return ppt == 1 ? 0 : ppt == 2 ? 1 : 2; }

// Predicted milliseconds of the batch (n sets of M[i] trajectories, N[i] steps).
double model_ms(const abp_ctx *ctx, const TuneTable &tt, int sched, int ppt, int64_t spl, int32_t n,
                const int64_t *M, const int64_t *N) {
    const float trial = tt.ms[sched][ppt_index(ppt)];
    if (!(trial < 1e29f)) return 1e300;
    const int64_t cap = candidate_capacity(ctx, sched, ppt);
    const bool ckpt = ctx->cfg.checkpoint_every > 0;
    const int64_t trial_traj = (int64_t)std::max(ctx->sm_count, 1) * kTrialTrajPerSm, trial_steps = kTrialSteps;
    const int64_t sms = std::max(ctx->sm_count, 1);
    const double eff_trial = batch_efficiency(1, &trial_traj, &trial_steps, sched, ppt, false,
                                              sched == 1 ? kTrialSteps : kTrialSteps / kTrialRounds, sms);
    const double eff = batch_efficiency(n, M, N, sched, ppt, ckpt, spl, sms);
    double work = 0.0;
    int64_t max_n = 0;
    for (int32_t i = 0; i < n; ++i) {
        work += (double)M[i] * (double)N[i];
        max_n = std::max(max_n, N[i]);
    }
    if (work <= 0.0) return 0.0;
    const double compute = (double)trial * eff_trial / std::max(eff, 1e-9) * work / ((double)trial_traj * trial_steps);
    const double sb = state_io_bytes(ctx->cfg);
    double bytes = 0.0, fixed = 0.0;
    if (sched == 1) {
        for (int64_t g = 0; g < max_n; g += spl) {
            double active = 0.0;
            for (int32_t i = 0; i < n; ++i)
                if (N[i] > g) active += (double)M[i];
            bytes += sb * active;
            fixed += kLaunchMs;
        }
    } else {
        const int64_t tile = (int64_t)kThreads * ppt;
        double items = 0.0;
        for (int32_t i = 0; i < n; ++i) {
            const double rounds = (double)((N[i] + spl - 1) / spl);
            bytes += sb * (double)M[i] * rounds;
            items += (double)((M[i] + tile - 1) / tile) * rounds;
        }
        fixed = kLaunchMs + items * kItemMs / (double)cap;
    }
    return compute + bytes / kHbmBytesPerMs + fixed;
}

// Round starts of the window [g0, g1): round j holds the tiles whose sets still
// have steps past g0 + j seg; since perm orders tiles by decreasing step count,
// those tiles are a prefix of perm.
std::vector<int32_t> round_starts(const abp_ctx *ctx, int64_t g0, int64_t g1, int64_t seg) {
    const int64_t n_rounds = (g1 - g0 + seg - 1) / seg;
    std::vector<int32_t> rs((size_t)n_rounds + 1, 0);
    int64_t cnt = ctx->n_tiles;  // tiles with n_steps > g0 + j seg
    int64_t acc = 0;
    for (int64_t j = 0; j < n_rounds; ++j) {
        const int64_t thr = g0 + j * seg;
        while (cnt > 0 && ctx->perm_steps[cnt - 1] <= thr) --cnt;
        rs[j] = (int32_t)acc;
        acc += cnt;
    }
    rs[n_rounds] = (int32_t)acc;
    return rs;
}

// The tiling, launch geometry and device tables of the current batch for one
// (schedule, trajectories per thread, steps per launch or per work item) choice,
// and the batch's initial condition drawn on the device.  Device buffers are
// reused when large enough.  Returns after the uploads have completed.
abp_status configure_batch(abp_ctx *ctx, int sched, int ppt, int64_t spl) {
    const int32_t n_sets = ctx->n_sets;
    ctx->sched = sched;
    ctx->ppt = ppt;
    ctx->g = 0;
    ctx->ckpt_complete = true;
    {
        TilePlan plan;
        if (!plan_tiles(n_sets, ctx->n_traj.data(), ctx->n_steps.data(), ctx->sched, ctx->ppt, ctx->cfg.checkpoint_every > 0, ctx->sm_count,
                        plan))
            return fail(ctx, ABP_EINVAL, "too many tiles");
        ctx->set_first.swap(plan.set_first);
        ctx->set_packed.swap(plan.set_packed);
        ctx->set_tile_begin.swap(plan.set_tile_begin);
        ctx->tile_first.swap(plan.tile_first);
        ctx->tile_count.swap(plan.tile_count);
        ctx->tile_set.swap(plan.tile_set);
        ctx->set_order.swap(plan.set_order);
        ctx->slot_set.swap(plan.slot_set);
        ctx->n_single = plan.n_single;
        ctx->n_tiles = (int32_t)ctx->tile_first.size();
        ctx->n_unpacked = plan.n_unpacked;
        ctx->narrow = plan.narrow;
        ctx->sub_single = plan.sub_single;
        ctx->sub_packed = plan.sub_packed;
    }
    const abp_config &c = ctx->cfg;
    const bool any_hist = c.hist_x_bins > 0 || c.hist_v_bins > 0;
    // snapshot slots: one per S steps when snapshot_every = S > 0 (histograms and live
    // results use them), else one final histogram snapshot when there are histograms
    ctx->n_snap = c.snapshot_every > 0 ? ctx->max_steps / c.snapshot_every : (any_hist ? 1 : 0);
    ctx->n_ckpt = c.checkpoint_every > 0 ? ctx->max_steps / c.checkpoint_every + 1 : 0;
    // Work-queue order: tiles by decreasing step count of their set (stable).
    ctx->perm.resize(ctx->n_tiles);
    for (int32_t t = 0; t < ctx->n_tiles; ++t) ctx->perm[t] = t;
    std::stable_sort(ctx->perm.begin(), ctx->perm.end(), [&](int32_t a, int32_t b) {
        return ctx->n_steps[ctx->tile_set[a]] > ctx->n_steps[ctx->tile_set[b]];
    });
    ctx->perm_steps.resize(ctx->n_tiles);
    for (int32_t k = 0; k < ctx->n_tiles; ++k) ctx->perm_steps[k] = ctx->n_steps[ctx->tile_set[ctx->perm[k]]];
    {
        int bps = 0;
        const size_t smem = sizeof(uint32_t) * (size_t)(std::max(c.hist_x_bins, 0) +
                                                        (c.hist_v_bins > 0 ? c.hist_v_bins + 2 : 0));
        cudaError_t oe =
            persistent_occupancy(c.state_fp64 != 0, ctx->ppt, smem, &bps, c.scheme == 1 ? 1 : c.noise == 1 ? 2 : 0);
        if (oe != cudaSuccess) return cuda_fail(ctx, oe, "occupancy query");
        ctx->grid = wq_blocks_per_sm(bps, ctx->n_tiles, ctx->sm_count) * std::max(ctx->sm_count, 1);
    }
    ctx->steps_per_launch = std::max<int64_t>(spl, 1);

    const size_t T = (size_t)ctx->total_traj;
    const size_t rsz = c.state_fp64 ? sizeof(double) : sizeof(float);
    abp_status st = ABP_OK;
#define ALLOC(buf, bytes, what) \
    if ((st = alloc(ctx, ctx->buf, (bytes), what)) != ABP_OK) { ctx->release_all(); return st; }
    ALLOC(d_params, sizeof(abp_params) * (size_t)n_sets, "parameters");
    ALLOC(d_coef, coef_table_bytes(n_sets), "step coefficients");
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
    if (c.noise == 1) ALLOC(d_xs, sizeof(uint4) * T, "xorshift states");
    ALLOC(d_hx, sizeof(uint32_t) * (size_t)ctx->n_snap * n_sets * (size_t)std::max(c.hist_x_bins, 0), "x histograms");
    ALLOC(d_hv, sizeof(uint32_t) * (size_t)ctx->n_snap * n_sets * (size_t)(c.hist_v_bins > 0 ? c.hist_v_bins + 2 : 0),
          "v histograms");
    ALLOC(d_ckpt, sizeof(float4) * (size_t)ctx->n_ckpt * T, "checkpoints");
    ALLOC(d_partials, sizeof(double) * 4 * (size_t)std::max(ctx->n_tiles, 1), "reduction scratch");
    ALLOC(d_moments, sizeof(double) * 8 * (size_t)std::max(n_sets, 1), "moments");
    ALLOC(d_queue, sizeof(int32_t) * ((size_t)ctx->n_tiles + 1), "work queue");
    ALLOC(d_perm, sizeof(int32_t) * (size_t)std::max(ctx->n_tiles, 1), "work queue order");
    ALLOC(d_set_first, sizeof(int64_t) * ((size_t)n_sets + 1), "set offsets");
    ALLOC(d_set_order, sizeof(int32_t) * (size_t)std::max(n_sets, 1), "set order");
    ALLOC(d_slot_set, sizeof(int32_t) * std::max(ctx->slot_set.size(), (size_t)1), "packed slot sets");
#undef ALLOC

    cudaStream_t s = ctx->stream;
    // The tables go up from one page-locked staging buffer (each piece at a 16-byte
    // offset); if it cannot be had, straight from the context's pageable vectors.
    const size_t stage_need = (sizeof(abp_params) * n_sets + 15) / 16 * 16 + (sizeof(int64_t) * n_sets + 15) / 16 * 16 +
                              (sizeof(int32_t) * (n_sets + 1) + 15) / 16 * 16 +
                              (sizeof(int64_t) * ctx->n_tiles + 15) / 16 * 16 +
                              3 * ((sizeof(int32_t) * ctx->n_tiles + 15) / 16 * 16) +
                              (sizeof(int64_t) * (n_sets + 1) + 15) / 16 * 16 + (sizeof(int32_t) * n_sets + 15) / 16 * 16 +
                              (sizeof(int32_t) * ctx->slot_set.size() + 15) / 16 * 16;
    if (ctx->h_stage_cap < stage_need) {
        if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
        ctx->h_stage = nullptr;
        ctx->h_stage_cap = 0;
        if (cudaMallocHost(&ctx->h_stage, stage_need) == cudaSuccess) {
            ctx->h_stage_cap = stage_need;
        } else {
            ctx->h_stage = nullptr;
            cudaGetLastError();
        }
    }
    size_t stage_off = 0;
    auto up = [&](DevBuf &b, const void *src, size_t n) -> cudaError_t {
        if (!n) return cudaSuccess;
        if (ctx->h_stage) {
            char *dst = (char *)ctx->h_stage + stage_off;
            memcpy(dst, src, n);
            stage_off += (n + 15) / 16 * 16;
            src = dst;
        }
        return cudaMemcpyAsync(b.p, src, n, cudaMemcpyHostToDevice, s);
    };
    cudaError_t e = up(ctx->d_params, ctx->params.data(), sizeof(abp_params) * n_sets);
    if (e == cudaSuccess) e = up(ctx->d_steps, ctx->n_steps.data(), sizeof(int64_t) * n_sets);
    if (e == cudaSuccess) e = up(ctx->d_set_tile_begin, ctx->set_tile_begin.data(), sizeof(int32_t) * (n_sets + 1));
    if (e == cudaSuccess) e = up(ctx->d_tile_first, ctx->tile_first.data(), sizeof(int64_t) * ctx->n_tiles);
    if (e == cudaSuccess) e = up(ctx->d_tile_count, ctx->tile_count.data(), sizeof(int32_t) * ctx->n_tiles);
    if (e == cudaSuccess) e = up(ctx->d_tile_set, ctx->tile_set.data(), sizeof(int32_t) * ctx->n_tiles);
    if (e == cudaSuccess) e = up(ctx->d_perm, ctx->perm.data(), sizeof(int32_t) * ctx->n_tiles);
    if (e == cudaSuccess) e = up(ctx->d_set_first, ctx->set_first.data(), sizeof(int64_t) * (n_sets + 1));
    if (e == cudaSuccess) e = up(ctx->d_set_order, ctx->set_order.data(), sizeof(int32_t) * n_sets);
    if (e == cudaSuccess) e = up(ctx->d_slot_set, ctx->slot_set.data(), sizeof(int32_t) * ctx->slot_set.size());
    if (e == cudaSuccess)
        e = launch_coef((const abp_params *)ctx->d_params.p, n_sets, ctx->cfg.dt, ctx->d_coef.p, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status.p, 0, sizeof(int32_t), s);
    if (e == cudaSuccess && ctx->d_hx.bytes) e = cudaMemsetAsync(ctx->d_hx.p, 0, ctx->d_hx.bytes, s);
    if (e == cudaSuccess && ctx->d_hv.bytes) e = cudaMemsetAsync(ctx->d_hv.p, 0, ctx->d_hv.bytes, s);
    if (e == cudaSuccess) {
        e = launch_init(ctx->batch(), ctx->state(), ctx->hist(), ctx->ckpt(), ctx->noise(), s);
        ctx->launches += ctx->n_tiles > 0 ? 1 : 0;
    }
    // The staging buffer (or the context's vectors) must not change before the
    // uploads complete: wait for them.
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ctx->release_batch();
        return cuda_fail(ctx, e, "upload / initial condition");
    }
    return ABP_OK;
}


cudaError_t enqueue_window(abp_ctx *ctx, int64_t g0, int64_t g1, const int32_t *round_start, int32_t n_rounds,
                           int32_t n_items, int64_t *kernels);

// Enqueue the window [g0, g1) of the configured batch without graph capture (the
// work queue's round starts uploaded to the context's buffer).
abp_status enqueue_direct(abp_ctx *ctx, int64_t g0, int64_t g1) {
    std::vector<int32_t> rs;
    int32_t n_rounds = 0, n_items = 0;
    const int32_t *d_rs = nullptr;
    if (ctx->sched == 2) {
        rs = round_starts(ctx, g0, g1, ctx->steps_per_launch);
        n_rounds = (int32_t)rs.size() - 1;
        n_items = rs.back();
        if (n_items == 0) return ABP_OK;
        abp_status st = alloc(ctx, ctx->d_round, sizeof(int32_t) * rs.size(), "work-queue rounds");
        if (st != ABP_OK) return st;
        ABP_CUDA(ctx, cudaMemcpyAsync(ctx->d_round.p, rs.data(), sizeof(int32_t) * rs.size(), cudaMemcpyHostToDevice,
                                      ctx->stream),
                 "work-queue rounds upload");
        d_rs = (const int32_t *)ctx->d_round.p;
    }
    int64_t k = 0;
    ABP_CUDA(ctx, enqueue_window(ctx, g0, g1, d_rs, n_rounds, n_items, &k), "integrator launch");
    ctx->launches += k;
    return ABP_OK;
}

// The autotuner's choice for the current batch and how it was reached.
struct TuneChoice {
    int sched = 1, ppt = 1;
    int64_t spl = 1;
};

struct Candidate {
    int sched, ppt;
    int64_t spl;
    double model_ms;           // model prediction for the whole batch
    int64_t probe_steps = 0;   // length of its probe prefix
    double probe_ms = -1.0;    // measured time of the probe prefix (-1: not probed)
    double probe_model = 0.0;  // model prediction for the probe prefix
    double pred_ms = 0.0;      // prediction the choice used
};

// Choices already made, by batch and configuration, so that a batch set again (a
// benchmark loop, a resumed run) is not probed again.
std::mutex g_choice_mu;
std::map<std::pair<int, uint64_t>, std::pair<TuneChoice, std::string>> g_choices;

uint64_t choice_key(const abp_ctx *ctx) {
    // FNV-1a over 8-byte words (every field hashed is a multiple of 8 bytes)
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *q, size_t n) {
        const unsigned char *c = (const unsigned char *)q;
        for (size_t i = 0; i + 8 <= n; i += 8) {
            uint64_t w;
            memcpy(&w, c + i, 8);
            h ^= w;
            h *= 1099511628211ull;
            h ^= h >> 29;
        }
    };
    mix(ctx->params.data(), sizeof(abp_params) * ctx->params.size());
    mix(ctx->n_traj.data(), sizeof(int64_t) * ctx->n_traj.size());
    mix(ctx->n_steps.data(), sizeof(int64_t) * ctx->n_steps.size());
    const abp_config &c = ctx->cfg;
    const int64_t f[] = {c.state_fp64, c.hist_x_bins, c.hist_v_bins, c.snapshot_every, c.checkpoint_every > 0,
                         c.particles_per_thread, c.schedule, c.steps_per_launch, c.scheme, c.noise};
    mix(f, sizeof(f));
    return h;
}

// Steps of the probe prefix: about 8e9 particle-steps of the batch (several ms on a
// GB300; 1/64 of that for the FP64 state, which steps ~100x slower), 256 to 16,384
// steps, and never more than the longest set.
int64_t probe_steps(const abp_ctx *ctx) {
    const double per_step = (double)std::max<int64_t>(ctx->total_traj, 1);
    const double target = ctx->cfg.state_fp64 ? 8e9 / 64.0 : 8e9;
    int64_t P = (int64_t)std::ceil(target / per_step);
    P = std::min<int64_t>(std::max<int64_t>(P, 256), 16384);
    P = (P + 63) / 64 * 64;
    return std::min(P, ctx->max_steps);
}

// The probe prefix of one candidate: P steps, but a work-queue candidate is timed
// over at least four of its own items where that stays within 3e10 particle-steps
// (FP64 state: 1/64 of it), so that the rounds of a tile follow one another as in
// the whole run (load sweep, 512 tiles, items of 10^4 steps: over 1.6 rounds the
// prefix predicted 28.4 ms for a run that takes 26.8).
int64_t probe_steps_for(const abp_ctx *ctx, int sched, int64_t spl, int64_t P) {
    if (sched != 2) return P;
    const double budget = ctx->cfg.state_fp64 ? 3e10 / 64.0 : 3e10;
    const int64_t fit = (int64_t)(budget / (double)std::max<int64_t>(ctx->total_traj, 1));
    int64_t Pc = std::max(P, std::min(4 * spl, fit));
    Pc = (Pc + 63) / 64 * 64;
    return std::min(Pc, ctx->max_steps);
}

// Configure the batch for candidate c and time its first P steps on the device
// (after a warm-up window, so that kernel loading is not timed).
abp_status probe_candidate(abp_ctx *ctx, Candidate &c, int64_t P) {
    abp_status st = configure_batch(ctx, c.sched, c.ppt, std::min(c.spl, P));
    if (st != ABP_OK) return st;
    const int32_t hold = ctx->hold_tile;
    ctx->hold_tile = -1;
    cudaStream_t s = ctx->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) st = enqueue_direct(ctx, 0, std::min<int64_t>(P, 64));
    if (e == cudaSuccess && st == ABP_OK) {
        e = launch_init(ctx->batch(), ctx->state(), ctx->hist(), ctx->ckpt(), ctx->noise(), s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) st = enqueue_direct(ctx, 0, P);
        if (e == cudaSuccess && st == ABP_OK) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess && st == ABP_OK) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess && st == ABP_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) c.probe_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ctx->hold_tile = hold;
    if (e == cudaSuccess && st == ABP_OK) {
        int32_t status = 0;  // a probe whose bounded waits expired does not count
        if (cudaMemcpy(&status, ctx->d_status.p, sizeof(int32_t), cudaMemcpyDeviceToHost) == cudaSuccess && status)
            c.probe_ms = -1.0;
        cudaMemsetAsync(ctx->d_status.p, 0, sizeof(int32_t), s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        c.probe_ms = -1.0;
    }
    return st;
}

// The autotuner: every allowed (schedule, trajectories per thread, steps per launch
// in {10^3, 10^4, 10^5} up to the longest set) is ranked by the model; when both
// schedules are allowed, the best candidate of each is then timed on the first steps of
// this very batch (its tiles, parameters and step counts) and each prediction becomes
// that measured time scaled by the model's ratio of the whole batch to the prefix; the
// smaller wins.  The choice is kept per batch and configuration.
TuneChoice choose_configuration(abp_ctx *ctx) {
    const abp_config &c = ctx->cfg;
    TuneChoice tc;
    const int want_sched = c.schedule, want_ppt = c.particles_per_thread;
    std::vector<int64_t> spls;
    if (c.steps_per_launch > 0) {
        spls.push_back(c.steps_per_launch);
    } else {
        for (int64_t S : {1000, 10000, 100000}) {
            const int64_t v = std::max<int64_t>(1, std::min(S, ctx->max_steps));
            if (std::find(spls.begin(), spls.end(), v) == spls.end()) spls.push_back(v);
        }
    }
    if (want_sched && want_ppt && spls.size() == 1) {
        tc.sched = want_sched;
        tc.ppt = want_ppt;
        tc.spl = spls[0];
        ctx->tune_report = "{\"fixed\": true}";
        return tc;
    }
    const std::pair<int, uint64_t> key(ctx->device, choice_key(ctx));
    {
        std::lock_guard<std::mutex> lock(g_choice_mu);
        auto it = g_choices.find(key);
        if (it != g_choices.end()) {
            ctx->tune_report = it->second.second;
            return it->second.first;
        }
        if (load_choice(ctx, key.second, &tc.sched, &tc.ppt, &tc.spl)) {
            char buf[160];
            snprintf(buf, sizeof(buf), "{\"from_cache_file\": true, \"chosen\": {\"schedule\": %d, \"ppt\": %d, "
                     "\"steps\": %lld}}", tc.sched, tc.ppt, (long long)tc.spl);
            ctx->tune_report = buf;
            g_choices[key] = std::make_pair(tc, ctx->tune_report);
            return tc;
        }
    }
    const int dev = ctx->device, kind = tune_kind(ctx);
    TuneTable local;
    TuneTable &tt = (dev >= 0 && dev < 64) ? g_tune[dev][kind] : local;
    if (!tt.done && !load_tune(ctx, tt)) {
        measure_candidates(ctx, tt);
        if (tt.done) save_tune(ctx, tt);
    }
    std::vector<Candidate> cands;
    for (int sch = 1; sch <= 2; ++sch) {
        if (want_sched && sch != want_sched) continue;
        for (int ppt : {1, 2, 4}) {
            if (want_ppt && ppt != want_ppt) continue;
            for (int64_t spl : spls) {
                Candidate cd{sch, ppt, spl, 0.0};
                cd.model_ms = model_ms(ctx, tt, sch, ppt, spl, ctx->n_sets, ctx->n_traj.data(), ctx->n_steps.data());
                cd.pred_ms = cd.model_ms;
                if (cd.model_ms < 1e299) cands.push_back(cd);
            }
        }
    }
    if (cands.empty()) cands.push_back(Candidate{want_sched ? want_sched : 1, want_ppt ? want_ppt : 1, spls[0], 0.0});
    // the best candidate of each schedule by the model
    int best_of[3] = {-1, -1, -1};
    for (int i = 0; i < (int)cands.size(); ++i) {
        int &b = best_of[cands[i].sched];
        if (b < 0 || cands[i].model_ms < cands[b].model_ms) b = i;
    }
    const int64_t P = probe_steps(ctx);
    const bool probe = best_of[1] >= 0 && best_of[2] >= 0 && ctx->total_traj > 0 && P > 0;
    std::vector<char> probed(cands.size(), 0);
    if (probe) {
        // probed: every candidate within kProbeBand of its schedule's best by the model (the
        // model cannot see everything a batch does to a kernel, so near-ties are measured);
        // candidates whose prefix runs the same launches (items or windows capped at the
        // prefix) share one measurement
        for (int i = 0; i < (int)cands.size(); ++i) {
            Candidate &cd = cands[i];
            if (cd.model_ms > cands[best_of[cd.sched]].model_ms * (1.0 + kProbeBand)) continue;
            probed[i] = 1;
            const int64_t Pc = probe_steps_for(ctx, cd.sched, cd.spl, P);
            cd.probe_steps = Pc;
            std::vector<int64_t> Np(ctx->n_steps);
            for (int64_t &v : Np) v = std::min(v, Pc);
            cd.probe_model = model_ms(ctx, tt, cd.sched, cd.ppt, std::min(cd.spl, Pc), ctx->n_sets,
                                      ctx->n_traj.data(), Np.data());
            for (int j = 0; j < i; ++j)
                if (probed[j] && cands[j].sched == cd.sched && cands[j].ppt == cd.ppt &&
                    cands[j].probe_steps == Pc && std::min(cands[j].spl, Pc) == std::min(cd.spl, Pc))
                    cd.probe_ms = cands[j].probe_ms;
            if (cd.probe_ms < 0.0 && probe_candidate(ctx, cd, Pc) != ABP_OK) cd.probe_ms = -1.0;
            if (cd.probe_ms > 0.0 && cd.probe_model > 0.0) cd.pred_ms = cd.probe_ms * cd.model_ms / cd.probe_model;
        }
        // a candidate whose probe failed is not chosen over one that was measured
        bool any_measured = false;
        for (int i = 0; i < (int)cands.size(); ++i) any_measured = any_measured || (probed[i] && cands[i].probe_ms > 0.0);
        for (int i = 0; i < (int)cands.size(); ++i)
            if (probed[i] && cands[i].probe_ms < 0.0 && any_measured) cands[i].pred_ms = 1e300;
    }
    int best = -1;
    for (int i = 0; i < (int)cands.size(); ++i) {
        if (probe && !probed[i]) continue;  // the probed candidates decide
        if (best < 0 || cands[i].pred_ms < cands[best].pred_ms) best = i;
    }
    tc.sched = cands[best].sched;
    tc.ppt = cands[best].ppt;
    tc.spl = cands[best].spl;
    std::string rep = "{\"probe_steps\": " + std::to_string(probe ? P : 0) + ", \"candidates\": [";
    char buf[256];
    for (size_t i = 0; i < cands.size(); ++i) {
        const Candidate &cd = cands[i];
        snprintf(buf, sizeof(buf),
                 "%s{\"schedule\": %d, \"ppt\": %d, \"steps\": %lld, \"model_ms\": %.4g, \"probe_steps\": %lld, "
                 "\"probe_ms\": %.4g, \"predicted_ms\": %.4g}",
                 i ? ", " : "", cd.sched, cd.ppt, (long long)cd.spl, cd.model_ms, (long long)cd.probe_steps, cd.probe_ms,
                 cd.pred_ms);
        rep += buf;
    }
    snprintf(buf, sizeof(buf), "], \"chosen\": {\"schedule\": %d, \"ppt\": %d, \"steps\": %lld}}", tc.sched, tc.ppt,
             (long long)tc.spl);
    rep += buf;
    ctx->tune_report = rep;
    {
        std::lock_guard<std::mutex> lock(g_choice_mu);
        g_choices[key] = std::make_pair(tc, rep);
        if (probe) save_choice(ctx, key.second, tc.sched, tc.ppt, tc.spl);
    }
    return tc;
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
    const NvtxRange nvtx("abp_create");
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
    if (cfg->schedule < 0 || cfg->schedule > 2) return ABP_EINVAL;
    if (cfg->checkpoint_every > 0 && cfg->state_fp64) return ABP_EINVAL;  // adjoint runs on the FP32 path
    if (cfg->scheme != 0 && cfg->scheme != 1) return ABP_EINVAL;
    if (cfg->scheme == 1 && (cfg->state_fp64 || cfg->checkpoint_every > 0)) return ABP_EINVAL;  // FP32, no adjoint
    if (cfg->noise != 0 && cfg->noise != 1) return ABP_EINVAL;
    if (cfg->noise == 1 && (cfg->scheme != 0 || cfg->state_fp64 || cfg->checkpoint_every > 0)) return ABP_EINVAL;
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
    ctx->ppt = cfg->particles_per_thread;  // 0: autotuned by abp_set_params
    *out = ctx;
    return ABP_OK;
}

void abp_destroy(abp_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    ctx->release_all();
    ctx->release_streams();
    ctx->d_status.release();
    delete ctx;
}

abp_status abp_set_params(abp_ctx *ctx, int32_t n_sets, const abp_params *sets, const int64_t *n_traj,
                          const int64_t *n_steps) {
    const NvtxRange nvtx("abp_set_params");
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
    ctx->ckpt_complete = true;

    const TuneChoice tc = choose_configuration(ctx);
    const abp_status st = configure_batch(ctx, tc.sched, tc.ppt, tc.spl);
    if (st != ABP_OK) return st;
    ctx->have_batch = true;
    return ABP_OK;
}

abp_status abp_reset(abp_ctx *ctx, uint64_t seed) {
    const NvtxRange nvtx("abp_reset");
    if (!ctx) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_reset before abp_set_params");
    ctx->cfg.seed = seed;
    ctx->g = 0;
    ctx->ckpt_complete = true;
    ctx->adj_valid = false;
    if (ctx->live_stream) cudaStreamSynchronize(ctx->live_stream);  // copies of the previous run end first
    ctx->live_sent = ctx->live_ready = 0;
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemsetAsync(ctx->d_status.p, 0, sizeof(int32_t), s);
    if (e == cudaSuccess && ctx->d_hx.bytes) e = cudaMemsetAsync(ctx->d_hx.p, 0, ctx->d_hx.bytes, s);
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

}  // extern "C"

namespace {

Queue make_queue(abp_ctx *ctx, const int32_t *round_start, int32_t n_rounds, int32_t n_items) {
    Queue q;
    q.head = (int32_t *)ctx->d_queue.p;
    q.done = (int32_t *)ctx->d_queue.p + 1;
    q.status = (int32_t *)ctx->d_status.p;
    q.round_start = round_start;
    q.perm = (const int32_t *)ctx->d_perm.p;
    q.n_rounds = n_rounds;
    q.n_items = n_items;
    q.hold_tile = ctx->hold_tile;
    q.wait_limit_ns = ctx->wait_limit_ns;
    return q;
}

// Enqueue the window [g0, g1) on the context's stream: lockstep launches of at
// most steps_per_launch steps each, or one work-queue launch whose round starts
// are read from `round_start`.  Returns the number of kernels enqueued.
cudaError_t enqueue_window(abp_ctx *ctx, int64_t g0, int64_t g1, const int32_t *round_start, int32_t n_rounds,
                           int32_t n_items, int64_t *kernels) {
    cudaStream_t s = ctx->stream;
    const Batch b = ctx->batch();
    const State st = ctx->state();
    const Hist h = ctx->hist();
    const Ckpt c = ctx->ckpt();
    const Noise nz = ctx->noise();
    *kernels = 0;
    if (ctx->sched == 1) {
        for (int64_t g = g0; g < g1; g += ctx->steps_per_launch) {
            const WaitCtl wc{(int32_t *)ctx->d_status.p, ctx->wait_limit_ns, ctx->hold_tile};
            cudaError_t e =
                launch_integrate(b, st, h, c, nz, ctx->ppt, g, std::min(g1, g + ctx->steps_per_launch), s, &wc);
            if (e != cudaSuccess) return e;
            *kernels += (b.n_single > 0 ? 1 : 0) + (b.n_tiles > b.n_single ? 1 : 0);
        }
        return cudaSuccess;
    }
    if (n_items == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(ctx->d_queue.p, 0, sizeof(int32_t) * ((size_t)ctx->n_tiles + 1), s);
    if (e != cudaSuccess) return e;
    const Queue q = make_queue(ctx, round_start, n_rounds, n_items);
    const int grid = (int)std::min<int64_t>(ctx->grid, n_items);
    e = launch_persistent(b, st, h, c, nz, q, ctx->ppt, grid, g0, g1, ctx->steps_per_launch, s);
    *kernels = 1;
    return e;
}

// Run the window [g0, g1).  A window met for the second time (same schedule,
// step range, seed and test settings) is captured into a CUDA graph, which is
// replayed from then on; work-queue graphs keep their round starts in a buffer
// of their own.
abp_status run_window(abp_ctx *ctx, int64_t g0, int64_t g1) {
    cudaStream_t s = ctx->stream;
    const int64_t seg = ctx->steps_per_launch;
    const uint64_t traj_base = ctx->cfg.traj_base, seed = ctx->cfg.seed;
    for (abp_ctx::GraphEntry &ge : ctx->graphs)
        if (ge.sched == ctx->sched && ge.g0 == g0 && ge.g1 == g1 && ge.seg == seg && ge.seed == seed &&
            ge.traj_base == traj_base && ge.hold == ctx->hold_tile && ge.wait_limit_ns == ctx->wait_limit_ns) {
            cudaError_t e = cudaGraphLaunch(ge.exec, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "graph replay");
            ctx->launches += ge.kernels;
            return ABP_OK;
        }
    std::vector<int32_t> rs;
    int32_t n_rounds = 0;
    int64_t n_items = 0;
    if (ctx->sched == 2) {
        rs = round_starts(ctx, g0, g1, seg);
        n_rounds = (int32_t)rs.size() - 1;
        n_items = rs.back();
        if (n_items == 0) return ABP_OK;
        if (n_items > INT32_MAX / 2) return fail(ctx, ABP_EINVAL, "too many work items; raise steps_per_launch");
    }
    // windows are remembered only while a graph may still be captured, and at most 4,096
    // of them (a caller stepping a few steps at a time meets millions of windows)
    bool seen = false;
    if (ctx->graphs.size() < 8) {
        const std::pair<int64_t, int64_t> win(g0, g1);
        seen = ctx->windows_seen.count(win) > 0;
        if (!seen) {
            if (ctx->windows_seen.size() >= 4096) ctx->windows_seen.clear();
            ctx->windows_seen.insert(win);
        }
    }
    if (s != nullptr && seen && ctx->graphs.size() < 8) {
        abp_ctx::GraphEntry ge{ctx->sched, 0, g0, g1, seg, seed, traj_base, ctx->hold_tile, ctx->wait_limit_ns,
                               (int32_t)n_items, nullptr, nullptr};
        cudaError_t e = cudaSuccess;
        if (ctx->sched == 2) {
            e = cudaMalloc(&ge.round_start, sizeof(int32_t) * rs.size());
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(ge.round_start, rs.data(), sizeof(int32_t) * rs.size(), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t le = enqueue_window(ctx, g0, g1, (const int32_t *)ge.round_start, n_rounds,
                                                  (int32_t)n_items, &ge.kernels);
            e = cudaStreamEndCapture(s, &graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess) {
            ctx->graphs.push_back(ge);
            e = cudaGraphLaunch(ge.exec, s);
            ctx->launches += ge.kernels;
            return e == cudaSuccess ? ABP_OK : cuda_fail(ctx, e, "graph launch");
        }
        // capture failed: fall back to direct launches
        cudaGetLastError();
        if (ge.round_start) cudaFree(ge.round_start);
    }
    const int32_t *d_rs = nullptr;
    if (ctx->sched == 2) {
        abp_status stt = alloc(ctx, ctx->d_round, sizeof(int32_t) * rs.size(), "work-queue rounds");
        if (stt != ABP_OK) return stt;
        cudaError_t e =
            cudaMemcpyAsync(ctx->d_round.p, rs.data(), sizeof(int32_t) * rs.size(), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "work-queue rounds upload");
        d_rs = (const int32_t *)ctx->d_round.p;
    }
    int64_t k = 0;
    const cudaError_t e = enqueue_window(ctx, g0, g1, d_rs, n_rounds, (int32_t)n_items, &k);
    ctx->launches += k;
    return e == cudaSuccess ? ABP_OK : cuda_fail(ctx, e, "integrator launch");
}

// Live results: the moments at step (k + 1) S on the device, then snapshot k's
// moments and histogram rows copied to the caller's page-locked buffers on the
// live stream, which waits for the main stream to reach this point.  Up to
// kLiveRing snapshots may be in flight; an older one is waited for first.
abp_status send_snapshot(abp_ctx *ctx, int64_t k) {
    cudaStream_t s = ctx->stream, ls = ctx->live_stream;
    const int R = abp_ctx::kLiveRing;
    const int slot = (int)(k % R);
    cudaError_t e = cudaSuccess;
    if (k - ctx->live_ready >= R) {  // the ring slot still belongs to snapshot k - R
        e = cudaEventSynchronize(ctx->live_copied[slot]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "live copy");
        ctx->live_ready = k - R + 1;
    }
    const size_t ns = (size_t)ctx->n_sets;
    double *dmom = ctx->live_mom ? (double *)ctx->d_live_mom.p + (size_t)k * ns * 8 : nullptr;
    if (dmom) {
        e = launch_reduce(ctx->batch(), ctx->state(), ctx->noise(), ctx->g, (double *)ctx->d_partials.p, dmom, s);
        ctx->launches += (ctx->n_sets > 0 && ctx->n_single > 0 ? 1 : 0) + (ctx->n_unpacked > 0 ? 1 : 0) +
                         (ctx->n_sets > ctx->n_unpacked ? 1 : 0);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->live_done[slot], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ls, ctx->live_done[slot], 0);
    if (e == cudaSuccess && dmom)
        e = cudaMemcpyAsync(ctx->live_mom + (size_t)k * ns * 8, dmom, sizeof(double) * 8 * ns, cudaMemcpyDeviceToHost,
                            ls);
    const size_t bx = (size_t)ctx->cfg.hist_x_bins, bv = ctx->cfg.hist_v_bins > 0 ? (size_t)ctx->cfg.hist_v_bins + 2 : 0;
    if (e == cudaSuccess && ctx->live_hx)
        e = cudaMemcpyAsync(ctx->live_hx + (size_t)k * ns * bx, (const uint32_t *)ctx->d_hx.p + (size_t)k * ns * bx,
                            sizeof(uint32_t) * ns * bx, cudaMemcpyDeviceToHost, ls);
    if (e == cudaSuccess && ctx->live_hv)
        e = cudaMemcpyAsync(ctx->live_hv + (size_t)k * ns * bv, (const uint32_t *)ctx->d_hv.p + (size_t)k * ns * bv,
                            sizeof(uint32_t) * ns * bv, cudaMemcpyDeviceToHost, ls);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->live_copied[slot], ls);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "live snapshot");
    ctx->live_sent = k + 1;
    return ABP_OK;
}

}  // namespace

extern "C" {

abp_status abp_integrate(abp_ctx *ctx, int64_t max_steps) {
    const NvtxRange nvtx("abp_integrate");
    if (!ctx) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_integrate before abp_set_params");
    const int64_t target = max_steps < 0 ? ctx->max_steps : std::min(ctx->max_steps, ctx->g + max_steps);
    if (target <= ctx->g) return ABP_OK;
    if (!ctx->live) {
        const abp_status st = run_window(ctx, ctx->g, target);
        if (st != ABP_OK) return st;
        ctx->g = target;
        return ABP_OK;
    }
    // live results: windows end at the snapshot steps, each followed by its snapshot's copy
    const int64_t S = ctx->cfg.snapshot_every;
    while (ctx->g < target) {
        const int64_t end = std::min(target, (ctx->g / S + 1) * S);
        abp_status st = run_window(ctx, ctx->g, end);
        if (st != ABP_OK) return st;
        ctx->g = end;
        if (end % S == 0 && end / S - 1 < ctx->n_snap && end / S - 1 == ctx->live_sent)
            if ((st = send_snapshot(ctx, end / S - 1)) != ABP_OK) return st;
    }
    return ABP_OK;
}

abp_status abp_live(abp_ctx *ctx, double *moments, uint32_t *hist_x, uint32_t *hist_v) {
    const NvtxRange nvtx("abp_live");
    if (!ctx) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_live before abp_set_params");
    if (ctx->live_stream) {
        cudaError_t e = cudaStreamSynchronize(ctx->live_stream);  // copies into the previous buffers end first
        if (e != cudaSuccess) return cuda_fail(ctx, e, "live stream synchronise");
    }
    if (!moments && !hist_x && !hist_v) {
        ctx->live = false;
        ctx->live_mom = nullptr;
        ctx->live_hx = ctx->live_hv = nullptr;
        return ABP_OK;
    }
    if (ctx->cfg.snapshot_every <= 0) return fail(ctx, ABP_EINVAL, "abp_live needs snapshot_every > 0");
    if (hist_x && ctx->cfg.hist_x_bins <= 0) return fail(ctx, ABP_EINVAL, "abp_live: hist_x given, hist_x_bins = 0");
    if (hist_v && ctx->cfg.hist_v_bins <= 0) return fail(ctx, ABP_EINVAL, "abp_live: hist_v given, hist_v_bins = 0");
    for (const void *p : {(const void *)moments, (const void *)hist_x, (const void *)hist_v}) {
        if (!p) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return fail(ctx, ABP_EINVAL, "abp_live: buffers must be page-locked host memory");
        }
    }
    cudaError_t e = cudaSuccess;
    if (!ctx->live_stream) {
        e = cudaStreamCreateWithFlags(&ctx->live_stream, cudaStreamNonBlocking);
        for (int i = 0; e == cudaSuccess && i < abp_ctx::kLiveRing; ++i) {
            e = cudaEventCreateWithFlags(&ctx->live_done[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->live_copied[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            ctx->release_streams();
            return cuda_fail(ctx, e, "live stream set-up");
        }
    }
    if (moments) {
        const abp_status st =
            alloc(ctx, ctx->d_live_mom, sizeof(double) * 8 * (size_t)std::max<int64_t>(ctx->n_snap, 1) *
                                            (size_t)std::max(ctx->n_sets, 1), "live moments");
        if (st != ABP_OK) return st;
    }
    ctx->live = true;
    ctx->live_mom = moments;
    ctx->live_hx = hist_x;
    ctx->live_hv = hist_v;
    ctx->live_sent = ctx->live_ready = std::min(ctx->g / ctx->cfg.snapshot_every, ctx->n_snap);
    return ABP_OK;
}

abp_status abp_live_ready(abp_ctx *ctx, int64_t *n_ready) {
    if (!ctx || !n_ready) return ABP_EINVAL;
    while (ctx->live && ctx->live_ready < ctx->live_sent) {
        const cudaError_t e = cudaEventQuery(ctx->live_copied[ctx->live_ready % abp_ctx::kLiveRing]);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "live copy");
        ++ctx->live_ready;
    }
    *n_ready = ctx->live_ready;
    return ABP_OK;
}

namespace {
bool plan_args_ok(int32_t n_sets, const int64_t *n_traj, const int64_t *n_steps, int32_t schedule, int32_t ppt) {
    if (n_sets < 0 || (n_sets > 0 && (!n_traj || !n_steps))) return false;
    if (schedule != 1 && schedule != 2) return false;
    if (ppt != 1 && ppt != 2 && ppt != 4) return false;
    for (int32_t i = 0; i < n_sets; ++i)
        if (n_traj[i] < 0 || n_steps[i] < 0) return false;
    return true;
}
}  // namespace

abp_status abp_plan(int32_t n_sets, const int64_t *n_traj, const int64_t *n_steps, int32_t schedule,
                    int32_t particles_per_thread, int32_t checkpoints, int32_t sm_count, int32_t *n_tiles,
                    int32_t *n_packed, int32_t *narrow, int64_t *tile_first, int32_t *tile_count, int32_t *tile_set,
                    int32_t max_tiles) {
    if (!plan_args_ok(n_sets, n_traj, n_steps, schedule, particles_per_thread) || sm_count < 1) return ABP_EINVAL;
    TilePlan p;
    if (!plan_tiles(n_sets, n_traj, n_steps, schedule, particles_per_thread, checkpoints != 0, sm_count, p))
        return ABP_EINVAL;
    const int32_t nt = (int32_t)p.tile_first.size();
    if (n_tiles) *n_tiles = nt;
    if (n_packed) *n_packed = nt - p.n_single;
    if (narrow) *narrow = p.narrow;
    if (max_tiles >= nt)
        for (int32_t t = 0; t < nt; ++t) {
            if (tile_first) tile_first[t] = p.tile_first[t];
            if (tile_count) tile_count[t] = p.tile_count[t];
            if (tile_set) tile_set[t] = p.tile_set[t];
        }
    return ABP_OK;
}

abp_status abp_plan_efficiency(int32_t n_sets, const int64_t *n_traj, const int64_t *n_steps, int32_t schedule,
                               int32_t particles_per_thread, int32_t checkpoints, int64_t steps_per_launch,
                               int64_t units, double *efficiency) {
    if (!efficiency || !plan_args_ok(n_sets, n_traj, n_steps, schedule, particles_per_thread) || units < 1 ||
        steps_per_launch < 0)
        return ABP_EINVAL;
    int64_t total = 0, max_n = 0;
    for (int32_t i = 0; i < n_sets; ++i) {
        total += n_traj[i];
        max_n = std::max(max_n, n_steps[i]);
    }
    const int64_t spl = steps_per_launch > 0 ? steps_per_launch : schedule == 1 ? default_window(total, max_n) : 0;
    *efficiency = batch_efficiency(n_sets, n_traj, n_steps, schedule, particles_per_thread, checkpoints != 0, spl,
                                   units);
    return ABP_OK;
}

abp_status abp_tiles(const abp_ctx *ctx, int32_t *n_tiles, int32_t *n_packed, int32_t *narrow) {
    if (!ctx) return ABP_EINVAL;
    if (n_tiles) *n_tiles = ctx->n_tiles;
    if (n_packed) *n_packed = ctx->n_tiles - ctx->n_single;
    if (narrow) *narrow = ctx->narrow;
    return ABP_OK;
}

abp_status abp_set_wait_limit(abp_ctx *ctx, int64_t wait_limit_ns) {
    if (!ctx || wait_limit_ns < 0) return ABP_EINVAL;
    ctx->wait_limit_ns = wait_limit_ns > 0 ? wait_limit_ns : 60000000000LL;
    return ABP_OK;
}

abp_status abp_test_hold_tile(abp_ctx *ctx, int32_t tile) {
    if (!ctx) return ABP_EINVAL;
    if (tile < -1 || (ctx->have_batch && tile >= ctx->n_tiles)) return fail(ctx, ABP_EINVAL, "tile out of range");
    ctx->hold_tile = tile;
    return ABP_OK;
}

abp_status abp_tuning(const abp_ctx *ctx, int32_t *schedule, int32_t *particles_per_thread, int64_t *steps_per_item,
                      int32_t *blocks) {
    if (!ctx) return ABP_EINVAL;
    if (schedule) *schedule = ctx->sched;
    if (particles_per_thread) *particles_per_thread = ctx->ppt;
    if (steps_per_item) *steps_per_item = ctx->steps_per_launch;
    if (blocks) {
        *blocks = ctx->grid;
        if (ctx->sched == 1) {  // lockstep: the blocks of the integrator resident at once
            const abp_config &c = ctx->cfg;
            const size_t smem =
                sizeof(uint32_t) * (size_t)(std::max(c.hist_x_bins, 0) + (c.hist_v_bins > 0 ? c.hist_v_bins + 2 : 0));
            int bps = 0;
            if (integrate_occupancy(c.state_fp64 != 0, ctx->ppt, smem, &bps, c.scheme == 1 ? 1 : c.noise == 1 ? 2 : 0) ==
                cudaSuccess)
                *blocks = bps * std::max(ctx->sm_count, 1);
            else
                cudaGetLastError();
        }
    }
    return ABP_OK;
}

abp_status abp_tuning_report(const abp_ctx *ctx, char *buf, size_t len, size_t *needed) {
    if (!ctx) return ABP_EINVAL;
    const std::string &r = ctx->tune_report;
    if (needed) *needed = r.size() + 1;
    if (buf && len) {
        const size_t n = std::min(len - 1, r.size());
        memcpy(buf, r.data(), n);
        buf[n] = '\0';
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
    const NvtxRange nvtx("abp_reduce");
    if (!ctx) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_reduce before abp_set_params");
    bool synced = false;
    abp_status st;
    if (moments) {
        // the kernels write every set's row: into a device output directly; into a small
        // page-locked host output through its device mapping (the call then waits for them:
        // measured 4 us faster per call than a copy for 64 sets, 6 us slower for 8,192, where
        // the copy engine moves the 512 KB faster than the kernels' stores); else into the
        // context's buffer, copied to the host
        const PtrKind k = ptr_kind(moments, ctx->device);
        if (k == PtrKind::OtherDevice)
            return fail(ctx, ABP_EINVAL, "an output points to another GPU's memory (the context runs on device %d)",
                        ctx->device);
        const size_t bytes = sizeof(double) * 8 * (size_t)ctx->n_sets;
        double *dst = k == PtrKind::Device ? moments : bytes <= 16384 ? mapped_host(moments) : nullptr;
        const bool copy = dst == nullptr;
        if (copy) dst = (double *)ctx->d_moments.p;
        if (k == PtrKind::Host && !copy) synced = true;
        cudaError_t e = launch_reduce(ctx->batch(), ctx->state(), ctx->noise(), ctx->g, (double *)ctx->d_partials.p,
                                      dst, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "reduction launch");
        ctx->launches += (ctx->n_sets > 0 && ctx->n_single > 0 ? 1 : 0) + (ctx->n_unpacked > 0 ? 1 : 0) +
                         (ctx->n_sets > ctx->n_unpacked ? 1 : 0);
        if (copy && (st = deliver(ctx, moments, ctx->d_moments.p, bytes, &synced)) != ABP_OK) return st;
    }
    if (hist_x && ctx->d_hx.bytes)
        if ((st = deliver(ctx, hist_x, ctx->d_hx.p, ctx->d_hx.bytes, &synced)) != ABP_OK) return st;
    if (hist_v && ctx->d_hv.bytes)
        if ((st = deliver(ctx, hist_v, ctx->d_hv.p, ctx->d_hv.bytes, &synced)) != ABP_OK) return st;
    if (synced) return abp_synchronize(ctx);
    return ABP_OK;
}

}  // extern "C"

namespace {

struct SaveHeader {
    char magic[8];  // "ABPSAVE1"
    uint32_t version, fp64;
    int64_t g, total_traj;
    int32_t n_sets, scheme;  // scheme: 0 Euler-Maruyama, 1 stochastic Heun
    uint64_t seed, traj_base;
    uint64_t hx_bytes, hv_bytes;
    uint64_t signature;  // FNV-1a of the sets' parameters, sizes and step counts
    int32_t noise, reserved;  // noise: 0 Philox, 1 xorshift (its states follow the cell indices)
};

uint64_t batch_signature(const abp_ctx *ctx) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *c = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    };
    mix(ctx->params.data(), sizeof(abp_params) * ctx->params.size());
    mix(ctx->n_traj.data(), sizeof(int64_t) * ctx->n_traj.size());
    mix(ctx->n_steps.data(), sizeof(int64_t) * ctx->n_steps.size());
    return h;
}

// The state arrays of an image, in order, with their sizes.
std::vector<std::pair<DevBuf *, size_t>> image_parts(abp_ctx *ctx) {
    const size_t T = (size_t)ctx->total_traj, rsz = ctx->cfg.state_fp64 ? sizeof(double) : sizeof(float);
    return {{&ctx->d_y, rsz * T},    {&ctx->d_yacc, rsz * T}, {&ctx->d_ylo, rsz * T},
            {&ctx->d_v, rsz * T},    {&ctx->d_e, rsz * T},    {&ctx->d_y0, rsz * T},
            {&ctx->d_cell, 4 * T},   {&ctx->d_xs, ctx->cfg.noise == 1 ? 16 * T : 0},
            {&ctx->d_hx, ctx->d_hx.bytes}, {&ctx->d_hv, ctx->d_hv.bytes}};
}

}  // namespace

extern "C" {

abp_status abp_save(abp_ctx *ctx, void *buf, size_t *bytes) {
    const NvtxRange nvtx("abp_save");
    if (!ctx || !bytes) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_save before abp_set_params");
    size_t need = sizeof(SaveHeader);
    for (auto &pt : image_parts(ctx)) need += pt.second;
    if (!buf) {
        *bytes = need;
        return ABP_OK;
    }
    if (*bytes < need) return fail(ctx, ABP_EINVAL, "abp_save: buffer of %zu bytes, %zu needed", *bytes, need);
    SaveHeader hd{};
    memcpy(hd.magic, "ABPSAVE1", 8);
    hd.version = 2;
    hd.noise = ctx->cfg.noise;
    hd.fp64 = ctx->cfg.state_fp64 ? 1 : 0;
    hd.g = ctx->g;
    hd.total_traj = ctx->total_traj;
    hd.n_sets = ctx->n_sets;
    hd.scheme = ctx->cfg.scheme;
    hd.seed = ctx->cfg.seed;
    hd.traj_base = ctx->cfg.traj_base;
    hd.hx_bytes = ctx->d_hx.bytes;
    hd.hv_bytes = ctx->d_hv.bytes;
    hd.signature = batch_signature(ctx);
    const PtrKind kind = ptr_kind(buf, ctx->device);
    if (kind == PtrKind::OtherDevice) return fail(ctx, ABP_EINVAL, "abp_save: buffer on another GPU");
    const bool dev = kind == PtrKind::Device;
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(buf, &hd, sizeof(hd), dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s);
    size_t off = sizeof(hd);
    for (auto &pt : image_parts(ctx)) {
        if (e == cudaSuccess && pt.second)
            e = cudaMemcpyAsync((char *)buf + off, pt.first->p, pt.second,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
        off += pt.second;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "abp_save");
    *bytes = need;
    return ABP_OK;
}

abp_status abp_load(abp_ctx *ctx, const void *buf, size_t bytes) {
    const NvtxRange nvtx("abp_load");
    if (!ctx || !buf) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_load before abp_set_params");
    SaveHeader hd{};
    if (bytes < sizeof(hd)) return fail(ctx, ABP_EINVAL, "abp_load: image too small");
    const PtrKind kind = ptr_kind(buf, ctx->device);
    if (kind == PtrKind::OtherDevice) return fail(ctx, ABP_EINVAL, "abp_load: image on another GPU");
    const bool dev = kind == PtrKind::Device;
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&hd, buf, sizeof(hd), dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "abp_load header");
    size_t need = sizeof(hd);
    for (auto &pt : image_parts(ctx)) need += pt.second;
    if (memcmp(hd.magic, "ABPSAVE1", 8) != 0 || hd.version != 2)
        return fail(ctx, ABP_EINVAL, "abp_load: not an image written by abp_save");
    if (hd.fp64 != (ctx->cfg.state_fp64 ? 1u : 0u) || hd.scheme != ctx->cfg.scheme || hd.noise != ctx->cfg.noise ||
        hd.total_traj != ctx->total_traj ||
        hd.n_sets != ctx->n_sets ||
        hd.signature != batch_signature(ctx) || hd.hx_bytes != ctx->d_hx.bytes || hd.hv_bytes != ctx->d_hv.bytes ||
        bytes < need || hd.g < 0 || hd.g > ctx->max_steps)
        return fail(ctx, ABP_EINVAL, "abp_load: the image belongs to a different batch or configuration");
    size_t off = sizeof(hd);
    for (auto &pt : image_parts(ctx)) {
        if (e == cudaSuccess && pt.second)
            e = cudaMemcpyAsync(pt.first->p, (const char *)buf + off, pt.second,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
        off += pt.second;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status.p, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "abp_load");
    ctx->g = hd.g;
    ctx->adj_valid = false;
    ctx->cfg.seed = hd.seed;
    ctx->cfg.traj_base = hd.traj_base;
    ctx->ckpt_complete = hd.g == 0;
    ctx->drop_graphs();
    return ABP_OK;
}

abp_status abp_get_state(abp_ctx *ctx, double *x, double *x0, double *v, double *e, double *vbar) {
    const NvtxRange nvtx("abp_get_state");
    if (!ctx) return ABP_EINVAL;
    if (!ctx->have_batch) return fail(ctx, ABP_ESTATE, "abp_get_state before abp_set_params");
    double *outs[5] = {x, x0, v, e, vbar};
    const size_t n = (size_t)ctx->total_traj;
    bool all_dev = true;
    for (double *p : outs) {
        if (!p) continue;
        const PtrKind k = ptr_kind(p, ctx->device);
        if (k == PtrKind::OtherDevice)
            return fail(ctx, ABP_EINVAL, "abp_get_state: an output points to another GPU's memory");
        if (k != PtrKind::Device) all_dev = false;
    }
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
    const NvtxRange nvtx("abp_synchronize");
    if (!ctx) return ABP_EINVAL;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && ctx->live_stream) e = cudaStreamSynchronize(ctx->live_stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronise");
    int32_t status = 0;
    e = cudaMemcpy(&status, ctx->d_status.p, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status readback");
    if (status == 1) return fail(ctx, ABP_ETIMEOUT, "a bounded device-side wait expired");
    if (status == 3) return fail(ctx, ABP_ESTATE, "an index check of the checked build failed on the device");
    if (status != 0) return fail(ctx, ABP_ESTATE, "device reported status %d", status);
    return ABP_OK;
}

abp_status abp_backward(abp_ctx *ctx, const double *dJ_dmean_v, double *grad);  // abp_adjoint.cu

abp_status abp_philox(uint64_t seed, const uint64_t *traj, const uint64_t *m, int64_t n, uint32_t *out,
                      void *cuda_stream) {
    if (n < 0) return ABP_EINVAL;
    if (n == 0) return ABP_OK;
    const int dev = current_device();
    if (!traj || !m || !out || ptr_kind(traj, dev) != PtrKind::Device || ptr_kind(m, dev) != PtrKind::Device ||
        ptr_kind(out, dev) != PtrKind::Device)
        return ABP_EINVAL;
    cudaError_t e = launch_philox((uint32_t)seed, (uint32_t)(seed >> 32), traj, m, n, out, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? ABP_OK : ABP_ECUDA;
}

abp_status abp_normals(uint64_t seed, uint64_t traj, uint64_t n0, int64_t count, float *out, void *cuda_stream) {
    if (count < 0) return ABP_EINVAL;
    if (count == 0) return ABP_OK;
    if (!out || ptr_kind(out, current_device()) != PtrKind::Device) return ABP_EINVAL;
    cudaError_t e = launch_normals((uint32_t)seed, (uint32_t)(seed >> 32), traj, n0, count, out,
                                   (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? ABP_OK : ABP_ECUDA;
}

abp_status abp_xorshift(uint64_t seed, uint64_t traj, int64_t count, uint32_t *out, void *cuda_stream) {
    if (count < 0) return ABP_EINVAL;
    if (count == 0) return ABP_OK;
    if (!out || ptr_kind(out, current_device()) != PtrKind::Device) return ABP_EINVAL;
    cudaError_t e = launch_xorshift((uint32_t)seed, (uint32_t)(seed >> 32), traj, count, out, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? ABP_OK : ABP_ECUDA;
}

abp_status abp_combine_moments(int32_t n_sets, double *moments, const int64_t *n_traj, const int64_t *n_steps,
                               double dt, void *cuda_stream) {
    const NvtxRange nvtx("abp_combine_moments");
    if (n_sets < 0 || !(dt > 0.0) || !std::isfinite(dt)) return ABP_EINVAL;
    if (n_sets == 0) return ABP_OK;
    if (!moments || !n_traj || !n_steps) return ABP_EINVAL;
    for (int32_t i = 0; i < n_sets; ++i)
        if (n_traj[i] < 0 || n_steps[i] < 0) return ABP_EINVAL;
    const PtrKind k = ptr_kind(moments, current_device());
    if (k == PtrKind::OtherDevice) return ABP_EINVAL;
    if (k == PtrKind::Device)
        return launch_combine_moments(n_sets, moments, n_traj, n_steps, dt, (cudaStream_t)cuda_stream) == cudaSuccess
                   ? ABP_OK
                   : ABP_ECUDA;
    for (int32_t i = 0; i < n_sets; ++i) {
        double *row = moments + (size_t)i * 8;
        const double a[4] = {row[4], row[5], row[6], row[7]};
        moments_from_sums(row, a, n_traj[i], n_steps[i], dt);
    }
    return ABP_OK;
}

}  // extern "C"
