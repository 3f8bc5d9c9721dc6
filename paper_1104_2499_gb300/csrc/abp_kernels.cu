// abp_kernels.cu -- sm_103a kernels of the ABP ensemble integrator
// (arXiv 1104.2499, Sec. 2, Fig. 1).
//
//   init_kernel       initial condition of every trajectory (Philox counter 2^63)
//   integrate_kernel  the hot loop: Philox4x32-10 -> Box-Muller -> Euler-Maruyama
//                     with the state in registers for thousands of steps,
//                     block-compensated position, shared-memory snapshot
//                     histograms and adjoint checkpoints
//   tile_reduce_kernel / set_reduce_kernel / packed_reduce_kernel
//                     fixed-order FP64 ensemble reduction (mean velocity,
//                     standard error, MSD, D_eff)
//   get_state_kernel  per-trajectory readback in FP64
//   philox_kernel / normals_kernel  raw noise for verification
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "abp_device.cuh"
#include "abp_internal.cuh"

// Minimum resident blocks per SM requested from the compiler for the
// integrator (bounds its register use); 0 leaves the choice to the compiler.
// Counter blocks (4 steps each) per iteration of the integrator's inner loop.
#ifndef ABP_GROUP_UNROLL
#define ABP_GROUP_UNROLL 2
#endif
// Warp-specialised narrow launches (noise drawn by producer warps); 0 keeps
// every narrow launch on the plain integrator.
#ifndef ABP_WS
#define ABP_WS 1
#endif
#ifndef ABP_MIN_BLOCKS
#define ABP_MIN_BLOCKS 0
#endif
#if ABP_MIN_BLOCKS > 0
#define ABP_INTEGRATE_BOUNDS __launch_bounds__(abp::kThreads, ABP_MIN_BLOCKS)
#else
#define ABP_INTEGRATE_BOUNDS __launch_bounds__(abp::kThreads)
#endif

namespace abp {

namespace {

constexpr int kGroupUnroll = ABP_GROUP_UNROLL;

template <typename R>
struct SV {
    R *y, *yacc, *ylo, *v, *e, *y0;
    int32_t *cell;
};

template <typename R>
__host__ __device__ SV<R> view(const State &s) {
    return SV<R>{(R *)s.y, (R *)s.yacc, (R *)s.ylo, (R *)s.v, (R *)s.e, (R *)s.y0, s.cell};
}

// Displacement in periods, x_n - x_0 = L * disp, accumulated in FP64.
template <typename R>
__device__ __forceinline__ double disp_periods(const SV<R> &s, int64_t t) {
    return (((double)s.cell[t] + (double)s.y[t]) + ((double)s.yacc[t] + (double)s.ylo[t])) - (double)s.y0[t];
}

// Set of the trajectory in slot li (< kThreads) of packed tile `tile`, from the
// table the host planner writes (one load instead of a search over the sets).
__device__ __forceinline__ int packed_set(const Batch &b, int tile, int li) {
    const int64_t i = dchk((int64_t)(tile - b.n_single) * kThreads + li, (int64_t)(b.n_tiles - b.n_single) * kThreads,
                           b.dbg);
    return (int)dchk(b.slot_set[i], b.n_sets, b.dbg);
}

// ---------------------------------------------------------------- snapshots

// Bin of the position fraction y (any real; wrapped here) into [0, bx).
template <typename R>
__device__ __forceinline__ int bin_x(R y, int bx) {
    const R yb = y - floor_r<R>(y);
    int b = (int)(yb * (R)bx);
    return b < bx ? (b < 0 ? 0 : b) : bx - 1;
}

// Bin of v: [0, bv) inside [v_lo, v_hi), bv for v < v_lo, bv + 1 for v >= v_hi.
template <typename R>
__device__ __forceinline__ int bin_v(R v, R v_lo, R v_hi, R scale, int bv) {
    if (!(v >= v_lo)) return bv;  // also catches NaN as underflow
    if (v >= v_hi) return bv + 1;
    int b = (int)((v - v_lo) * scale);
    return b < bv ? b : bv - 1;
}

// Barrier over the threads that step trajectories: the whole block, or in a
// warp-specialised block (WS) its first `n` threads, on hardware barrier 1.
template <bool WS>
__device__ __forceinline__ void stepper_barrier(int n) {
    if constexpr (WS)
        asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
    else
        __syncthreads();
}

// Add the block's counts to the global histogram of (snap, set) and clear
// the shared copy.  Must be reached by every stepping thread of the block
// (`n` of them: blockDim.x, or the consumer threads of a WS block).
template <bool WS = false>
__device__ __forceinline__ void flush_hist(uint32_t *sh, const Hist &h, int64_t snap, int32_t set, int32_t n_sets,
                                           int n = 0) {
    if constexpr (!WS) n = blockDim.x;
    stepper_barrier<WS>(n);
    const int nb = h.bx + (h.bv > 0 ? h.bv + 2 : 0);
    for (int i = threadIdx.x; i < nb; i += n) {
        const uint32_t c = sh[i];
        if (c) {
            if (i < h.bx)
                atomicAdd(&h.x[((size_t)snap * n_sets + set) * h.bx + i], c);
            else
                atomicAdd(&h.v[((size_t)snap * n_sets + set) * (h.bv + 2) + (i - h.bx)], c);
        }
        sh[i] = 0;
    }
    stepper_barrier<WS>(n);
}

// ---------------------------------------------------------------- init

template <typename R>
__global__ void __launch_bounds__(kThreads) init_kernel(Batch b, State st, Hist h, Ckpt ck, Noise nz) {
    extern __shared__ uint32_t sh[];
    const SV<R> s = view<R>(st);
    const int tile = blockIdx.x;
    const int set = b.tile_set[tile];
    const bool packed = tile >= b.n_single;  // several sets, one trajectory per thread
    const int64_t first = b.tile_first[tile];
    const int count = b.tile_count[tile];
    const bool snap0 = h.snap_every <= 0 && b.set_steps[set] == 0 && (h.bx > 0 || h.bv > 0);
    const int nb = h.bx + (h.bv > 0 ? h.bv + 2 : 0);
    if (snap0 && !packed) {
        for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
    for (int li = threadIdx.x; li < count; li += blockDim.x) {
        const int64_t t = dchk(first + li, b.total_traj, b.dbg);
        const int my_set = packed ? packed_set(b, tile, li) : set;
        const abp_params p = b.params[my_set];
        const uint4 w = noise_block(kInitCounter, (uint64_t)t + nz.traj_base, nz.k0, nz.k1);
        const R y0 = (R)(w.x >> 8) * (R)0x1p-24;
        R v0 = 0;
        if (nz.v0_mode == 1) {
            // FP64 Box-Muller for both state types, rounded once: the initial velocity is
            // the earliest perturbation a trajectory sees, so near an unstable point of
            // the potential an error of the FP32 fast path (~1e-6 relative) grows by two
            // orders of magnitude over 10^3 steps.  One transform per trajectory and run.
            double ze, zo;
            box_muller_f64(w.y, w.z, ze, zo);
            v0 = (R)(sqrt(p.D) * ze);
        }
        if (nz.noise == 1 && st.xs) st.xs[t] = xorshift_seed((uint64_t)t + nz.traj_base, nz.k0, nz.k1);
        s.y[t] = y0;
        s.y0[t] = y0;
        s.yacc[t] = 0;
        s.ylo[t] = 0;
        s.v[t] = v0;
        s.e[t] = 0;
        s.cell[t] = 0;
        if (ck.every > 0 && sizeof(R) == 4) ck.ck[t] = make_float4((float)y0, 0.0f, (float)v0, 0.0f);
        if (snap0) {
            const R lo = (R)h.v_lo, hi = (R)h.v_hi;
            if (!packed) {
                if (h.bx > 0) atomicAdd(&sh[bin_x<R>(y0, h.bx)], 1u);
                if (h.bv > 0) atomicAdd(&sh[h.bx + bin_v<R>(v0, lo, hi, (R)(h.bv / (h.v_hi - h.v_lo)), h.bv)], 1u);
            } else {
                if (h.bx > 0) atomicAdd(&h.x[(size_t)my_set * h.bx + bin_x<R>(y0, h.bx)], 1u);
                if (h.bv > 0)
                    atomicAdd(&h.v[(size_t)my_set * (h.bv + 2) +
                                   bin_v<R>(v0, lo, hi, (R)(h.bv / (h.v_hi - h.v_lo)), h.bv)],
                              1u);
            }
        }
    }
    if (snap0 && !packed) flush_hist(sh, h, 0, set, b.n_sets);
}

// ---------------------------------------------------------------- integrator



template <typename R, int PPT>
struct Slots {
    R y[PPT], yacc[PPT], ylo[PPT], v[PPT], e[PPT];
    float pb[PPT];  // phase_base(y) of the FP32 path
    int32_t cell[PPT];
    StepStream ss[PPT];
    uint32_t xs[PPT][4];  // xorshift states (mode 2)
};

// Integrator modes (template parameter MODE): 0 Euler-Maruyama with Philox
// noise, 1 stochastic Heun with Philox noise, 2 Euler-Maruyama with xorshift
// noise (two words and one Box-Muller cosine per step).
constexpr int kModeEM = 0, kModeHeun = 1, kModeXorshift = 2;

// Round keys of the launch's seed as a kernel parameter (constant bank).
struct KeyParam {
    RoundKeys K;
};

// The FP32 step of the configured scheme.
template <bool HEUN>
__device__ __forceinline__ void step_f32(const Coef<float> &k, float nrs, float trig, float pb, float &yacc, float &v,
                                         float &e) {
    if constexpr (HEUN)
        heun_step_f32(k, nrs, trig, pb, yacc, v, e);
    else
        em_step_f32(k, nrs, trig, pb, yacc, v, e);
}

// The paired FP32 step of the configured scheme (two trajectories).
template <bool HEUN>
__device__ __forceinline__ void step_f32x2(const Coef2 &k, float2 nrs, float2 trig, float2 pb, float2 &yacc,
                                           float2 &v, float2 &e) {
    if constexpr (HEUN)
        heun_step_f32x2(k, nrs, trig, pb, yacc, v, e);
    else
        em_step_f32x2(k, nrs, trig, pb, yacc, v, e);
}

// Slots 2p and 2p + 1 as FP32 pairs, and back.
template <int PPT>
struct Pair {
    float2 yacc, v, e, pb;
    __device__ __forceinline__ Pair(const Slots<float, PPT> &S, int p)
        : yacc(make_float2(S.yacc[p], S.yacc[p + 1])), v(make_float2(S.v[p], S.v[p + 1])),
          e(make_float2(S.e[p], S.e[p + 1])), pb(make_float2(S.pb[p], S.pb[p + 1])) {}
    __device__ __forceinline__ void store(Slots<float, PPT> &S, int p) const {
        S.yacc[p] = yacc.x;
        S.yacc[p + 1] = yacc.y;
        S.v[p] = v.x;
        S.v[p + 1] = v.y;
        S.e[p] = e.x;
        S.e[p + 1] = e.y;
    }
};

// Whether the FP32 slots of a thread are stepped in pairs.
template <typename R, int PPT>
constexpr bool kPaired = sizeof(R) == 4 && PPT % 2 == 0 && ABP_F32X2 && ABP_ANGLE_FFMA;

// One Euler-Maruyama step of every slot at an arbitrary step index n (the
// unaligned head / tail of a range): the counter block of n is generated for
// this step alone.
template <typename R, int PPT, int MODE = kModeEM>
__device__ __forceinline__ void single_step(const Coef<R> &k, const RoundKeys &K, Slots<R, PPT> &S, int64_t n) {
    if constexpr (MODE == kModeXorshift && kPaired<R, PPT>) {
        const Coef2 k2 = make_coef2(k);
#pragma unroll
        for (int p = 0; p < PPT; p += 2) {
            Pair<PPT> P(S, p);
            uint2 wa, wb;
            wa.x = xorshift128(S.xs[p]);
            wb.x = xorshift128(S.xs[p]);
            wa.y = xorshift128(S.xs[p + 1]);
            wb.y = xorshift128(S.xs[p + 1]);
            float2 nrs, cs, sn;
            box_muller_f32x2(wa, wb, k2.bm, nrs, cs, sn);
            em_step_f32x2(k2, nrs, cs, P.pb, P.yacc, P.v, P.e);
            P.store(S, p);
        }
        return;
    } else if constexpr (MODE == kModeXorshift) {
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            float nrs, cs, sn;
            const uint32_t wa = xorshift128(S.xs[q]);
            const uint32_t wb = xorshift128(S.xs[q]);
            box_muller_f32(wa, wb, k.bm, nrs, cs, sn);
            em_step_f32(k, nrs, cs, S.pb[q], S.yacc[q], S.v[q], S.e[q]);
        }
        return;
    }
    const uint32_t j = (uint32_t)(n & 3);
    const uint32_t m = (uint32_t)(n >> 2);
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const uint4 w = step_block(m, S.ss[q], K);
        if constexpr (sizeof(R) == 4) {
            float nrs, cs, sn;
            if (j < 2)
                box_muller_f32(w.x, w.y, k.bm, nrs, cs, sn);
            else
                box_muller_f32(w.z, w.w, k.bm, nrs, cs, sn);
            step_f32<MODE == kModeHeun>(k, nrs, (j & 1) ? sn : cs, S.pb[q], S.yacc[q], S.v[q], S.e[q]);
        } else {
            const double z = normal_from_block_f64(w, j);
            em_step<double>(k, k.sigma * z, S.y[q], S.yacc[q], S.v[q], S.e[q]);
        }
    }
}

// Four steps 4m .. 4m+3 of every slot from one counter block each.
template <typename R, int PPT, int MODE = kModeEM>
__device__ __forceinline__ void group_step(const Coef<R> &k, const RoundKeys &K, Slots<R, PPT> &S, uint32_t m) {
    if constexpr (MODE == kModeXorshift) {
#pragma unroll
        for (int i = 0; i < 4; ++i) single_step<R, PPT, MODE>(k, K, S, 0);
        return;
    }
    constexpr bool HEUN = MODE == kModeHeun;
    uint4 w[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) w[q] = step_block(m, S.ss[q], K);
    if constexpr (kPaired<R, PPT>) {
        // trajectories 2p and 2p + 1 in the two halves of FP32 register pairs
        const Coef2 k2 = make_coef2(k);
#pragma unroll
        for (int p = 0; p < PPT; p += 2) {
            Pair<PPT> P(S, p);
            float2 nr, cs, sn;
            box_muller_f32x2(make_uint2(w[p].x, w[p + 1].x), make_uint2(w[p].y, w[p + 1].y), k2.bm, nr, cs, sn);
            step_f32x2<HEUN>(k2, nr, cs, P.pb, P.yacc, P.v, P.e);
            step_f32x2<HEUN>(k2, nr, sn, P.pb, P.yacc, P.v, P.e);
            box_muller_f32x2(make_uint2(w[p].z, w[p + 1].z), make_uint2(w[p].w, w[p + 1].w), k2.bm, nr, cs, sn);
            step_f32x2<HEUN>(k2, nr, cs, P.pb, P.yacc, P.v, P.e);
            step_f32x2<HEUN>(k2, nr, sn, P.pb, P.yacc, P.v, P.e);
            P.store(S, p);
        }
    } else if constexpr (sizeof(R) == 4) {
        float nr[PPT], cs[PPT], sn[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) box_muller_f32(w[q].x, w[q].y, k.bm, nr[q], cs[q], sn[q]);
#pragma unroll
        for (int q = 0; q < PPT; ++q) step_f32<HEUN>(k, nr[q], cs[q], S.pb[q], S.yacc[q], S.v[q], S.e[q]);
#pragma unroll
        for (int q = 0; q < PPT; ++q) step_f32<HEUN>(k, nr[q], sn[q], S.pb[q], S.yacc[q], S.v[q], S.e[q]);
#pragma unroll
        for (int q = 0; q < PPT; ++q) box_muller_f32(w[q].z, w[q].w, k.bm, nr[q], cs[q], sn[q]);
#pragma unroll
        for (int q = 0; q < PPT; ++q) step_f32<HEUN>(k, nr[q], cs[q], S.pb[q], S.yacc[q], S.v[q], S.e[q]);
#pragma unroll
        for (int q = 0; q < PPT; ++q) step_f32<HEUN>(k, nr[q], sn[q], S.pb[q], S.yacc[q], S.v[q], S.e[q]);
    } else {
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            double z0, z1, z2, z3;
            box_muller_f64(w[q].x, w[q].y, z0, z1);
            box_muller_f64(w[q].z, w[q].w, z2, z3);
            em_step<double>(k, k.sigma * z0, S.y[q], S.yacc[q], S.v[q], S.e[q]);
            em_step<double>(k, k.sigma * z1, S.y[q], S.yacc[q], S.v[q], S.e[q]);
            em_step<double>(k, k.sigma * z2, S.y[q], S.yacc[q], S.v[q], S.e[q]);
            em_step<double>(k, k.sigma * z3, S.y[q], S.yacc[q], S.v[q], S.e[q]);
        }
    }
}

// Counter blocks per iteration of the inner loop, per kernel (measured): the
// lockstep FP32 Euler-Maruyama kernel with two trajectories per thread runs
// fastest with 8 blocks (32 steps) per iteration on the D x q sweep, 1.038e12
// against 1.011e12 particle-steps/s with 2 and 0.98e12 with 12 (a body that no
// longer fits the instruction cache).  The work-queue kernel takes 8 as well, at
// 92 registers and two blocks per SM: against 6 (the same registers), uneven
// batch 1.005e12 against 9.89e11, load sweep 9.95e11 against 9.83e11, D x q sweep
// 1.020e12 against 1.006e12; capped at 80 registers for three blocks per SM it
// spills and loses 8% on the load sweep.  The stochastic Heun kernel at two per
// thread takes 4 (D x q sweep 6.92e11 against 6.88e11 with 2 and 3).  The other
// kernels keep the default, where longer bodies cost registers and blocks per SM
// without a measured gain.
#ifndef ABP_UNROLL_EM2
#define ABP_UNROLL_EM2 8
#endif
#ifndef ABP_UNROLL_EM2_QUEUE
#define ABP_UNROLL_EM2_QUEUE 8
#endif
#ifndef ABP_UNROLL_HEUN2
#define ABP_UNROLL_HEUN2 4
#endif
template <typename R, int PPT, int MODE, bool QUEUE>
constexpr int group_unroll() {
    if constexpr (sizeof(R) == 4 && PPT == 2 && MODE == kModeEM)
        return QUEUE ? ABP_UNROLL_EM2_QUEUE : ABP_UNROLL_EM2;
    else if constexpr (sizeof(R) == 4 && PPT == 2 && MODE == kModeHeun)
        return ABP_UNROLL_HEUN2;
    else
        return kGroupUnroll;
}

// Steps [n, n_end) of every slot.  Folds happen after absolute multiples of
// kBlockSteps steps; counter blocks are absolute multiples of 4.
template <typename R, int PPT, int MODE = kModeEM, int UNROLL = kGroupUnroll>
__device__ __forceinline__ void advance(const Coef<R> &k, const RoundKeys &K, Slots<R, PPT> &S, int64_t n,
                                        int64_t n_end) {
    while (n < n_end) {
        const int64_t blk_end = min(n_end, (n | (int64_t)(kBlockSteps - 1)) + 1);
        while (n < blk_end && (n & 3)) {
            single_step<R, PPT, MODE>(k, K, S, n);
            ++n;
        }
        if (n < blk_end) {
            const uint32_t m_end = (uint32_t)(blk_end >> 2);
            uint32_t m = (uint32_t)(n >> 2);
#pragma unroll UNROLL
            for (; m < m_end; ++m) group_step<R, PPT, MODE>(k, K, S, m);
            n = (int64_t)m << 2;
        }
        while (n < blk_end) {
            single_step<R, PPT, MODE>(k, K, S, n);
            ++n;
        }
        if ((blk_end & (kBlockSteps - 1)) == 0) {
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                fold_position<R>(S.y[q], S.yacc[q], S.ylo[q], S.cell[q]);
                if constexpr (sizeof(R) == 4) S.pb[q] = phase_base(S.y[q]);
            }
        }
    }
}

// ------------------------------------------- warp-specialised narrow launch
// A narrow launch of 32-thread blocks puts fewer than two warps on an SM, so a
// warp steps alone and its time per step is the latency of its own chain: the counter
// block and Box-Muller of four steps, then four dependent state updates.  In
// the warp-specialised form a consumer warp (its 32 trajectories stepped as in
// run_tile) has NP producer warps that draw the same (nrs, trig) pairs for the
// same steps ahead into a shared-memory ring; the consumer's chain is the state
// update alone.  The ring holds kWsSlots slots of kWsSlotSteps steps; slot j of
// a launch holds absolute steps [j S, (j + 1) S), so a slot ends where a
// position fold does.  Producer p writes counter blocks p, p + NP, ... of each
// slot.  Hand-over is by counters in shared memory: filled[p] = slots of the
// launch producer p has written, consumed = slots the consumer has finished,
// each stored by one lane after a warp barrier with release semantics and read
// with acquire semantics.  The consumer checks once per slot and only when its
// last reading is used up; a check at a slot boundary costs it the drain of its
// dependent chain, so slots are long: with 16-step slots the checks took about
// 29 of 59 cycles per step, with 64-step slots about 4 of 34.
// Every wait is bounded: past the wait limit the thread records status 1 and
// stops waiting, so the launch runs to its end and the host reports the timeout.
constexpr int kWsSlotSteps = 64;
constexpr int kWsSlots = 3;
static_assert(kWsSlotSteps == kBlockSteps, "a slot ends where a fold does");
// Producer warps per consumer warp: with one block per SM each of the SM's four
// schedulers runs one warp, and three producers draw the noise faster than the
// consumer uses it (one producer warp alone: about 75 cycles per step).  Where a
// launch puts two blocks on an SM, three producers per block still beat one.
constexpr int kWsProducers = 3;
// Narrow launches planned at most this wide run warp-specialised, as 32-thread
// stepping blocks.  Measured on the work-items sweep (one-trajectory sets, 10^4
// steps per cycle): 2^14 items, planned 64 wide (256 blocks), 0.42 ms per cycle
// on the plain narrow kernel and 0.34 ms warp-specialised (512 blocks of four
// warps, all resident); at 2^15 (128 wide) the warp-specialised grid would no
// longer fit on the SMs at once.
#ifndef ABP_WS_WIDEST
#define ABP_WS_WIDEST 64
#endif

struct WsRing {
    float2 *buf;        // [kWsSlots][kWsSlotSteps][32] (nrs, trig) per lane and step
    int32_t *filled;    // [NP]: slots of the launch written by producer warp p
    int32_t *consumed;  // slots of the launch the consumer warp has finished
    int32_t *status;    // 1 once a wait gave up
    int64_t limit_ns;
    int32_t hold_tile;  // test hook: the producers of this tile never hand a slot over
};

// Publish a warp's count: every lane's shared-memory accesses before the call
// are ordered (warp barrier, then one release store) before the new value.
__device__ __forceinline__ void ws_publish(int32_t *cnt, int32_t v) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) st_release_cta(cnt, v);
}

// Wait until *cnt >= target, at most limit_ns; returns the last value read.
// After a failure (here or in another thread) the thread no longer waits.
__device__ __forceinline__ int32_t ws_wait(const int32_t *cnt, int32_t target, const WsRing &r, bool &failed) {
    int32_t v = ld_acquire_cta(cnt);
    if (v >= target || failed) return v;
    const uint64_t t0 = global_ns();
    for (;;) {
        v = ld_acquire_cta(cnt);
        if (v >= target) return v;
        if (*(volatile int32_t *)r.status != 0 || global_ns() - t0 > (uint64_t)r.limit_ns) {
            atomicCAS(r.status, 0, 1);
            failed = true;
            return v;
        }
    }
}

// Consumer side: the launch's first slot, the slots known to be written by
// every producer it waits on (1 with xorshift noise, whose generator only the
// first producer runs), and whether a wait gave up.
struct WsCons {
    WsRing r;
    int np;
    int64_t a0;
    int32_t ready;
    bool failed;
};

// advance() with the noise taken from the ring (FP32, one trajectory per
// thread; the producers drew it from the counter-based stream or from the
// trajectory's xorshift generator).
template <bool HEUN>
__device__ __forceinline__ void advance_ws(const Coef<float> &k, Slots<float, 1> &S, int64_t n, int64_t n_end,
                                           WsCons &c) {
    constexpr int SS = kWsSlotSteps;
    const int lane = threadIdx.x & 31;
    while (n < n_end) {
        const int64_t a = n / SS;
        const int32_t kf = (int32_t)(a - c.a0);
        if (kf >= c.ready) {
            int32_t rd = ws_wait(&c.r.filled[0], kf + 1, c.r, c.failed);
            for (int p = 1; p < c.np; ++p) rd = min(rd, ws_wait(&c.r.filled[p], kf + 1, c.r, c.failed));
            c.ready = c.failed ? INT32_MAX : rd;
        }
        const float2 *ring = c.r.buf + (size_t)(kf % kWsSlots) * SS * 32 + lane;
        const int64_t a_end = min(n_end, (a + 1) * SS);
        if (n == a * SS && a_end == (a + 1) * SS) {
#pragma unroll
            for (int i = 0; i < SS; ++i) {
                const float2 t = ring[i * 32];
                step_f32<HEUN>(k, t.x, t.y, S.pb[0], S.yacc[0], S.v[0], S.e[0]);
            }
        } else {
            for (; n < a_end; ++n) {
                const float2 t = ring[(int)(n - a * SS) * 32];
                step_f32<HEUN>(k, t.x, t.y, S.pb[0], S.yacc[0], S.v[0], S.e[0]);
            }
        }
        n = a_end;
        if ((n & (kBlockSteps - 1)) == 0) {  // the slot's last step: fold, and hand the slot back
            fold_position<float>(S.y[0], S.yacc[0], S.ylo[0], S.cell[0]);
            S.pb[0] = phase_base(S.y[0]);
            ws_publish(c.r.consumed, kf + 1);
        }
    }
}

// Steps [max(w0, 0), w1) ∩ [0, N) of every trajectory of one tile: load the
// state (through L2, so a tile continued by another block sees its latest
// state), step it in registers, fill snapshot histograms and checkpoints, and
// store it back.  Must be reached by every thread of the block; `sh` holds
// zeros on entry (when histograms are on) and on exit.
// PACKED: a packed tile (several sets of equal step count, PPT 1): each thread
// takes the coefficients of its own trajectory's set, and histograms go to
// global memory directly.
// WS: the consumer threads of a warp-specialised block (noise from the ring
// of `wc`, histogram flushes on the consumers' own barrier).
template <typename R, int PPT, bool PACKED = false, int MODE = kModeEM, int UNROLL = kGroupUnroll, bool WS = false>
__device__ __forceinline__ void run_tile(const Batch &b, const State &st, const Hist &h, const Ckpt &ck,
                                         const Noise &nz, const RoundKeys &K, uint32_t *sh, int tile, int64_t w0,
                                         int64_t w1, int lane_base = 0, WsCons *wc = nullptr) {
    static_assert(!PACKED || PPT == 1, "packed tiles hold one trajectory per thread");
    static_assert(!WS || (sizeof(R) == 4 && PPT == 1), "WS: FP32, one trajectory per thread");
    tile = (int)dchk(tile, b.n_tiles, b.dbg);
    const int64_t first = b.tile_first[tile];
    const int count = b.tile_count[tile];
    const int set_t = (int)dchk(b.tile_set[tile], b.n_sets, b.dbg);
    const int64_t N = b.set_steps[set_t];
    const int64_t n_begin = min(w0, N);
    const int64_t n_end = min(w1, N);
    if (n_begin >= n_end) return;  // uniform over the block

    const SV<R> s = view<R>(st);
    const int set =
        PACKED ? packed_set(b, tile, min(lane_base + (int)threadIdx.x, count - 1)) : set_t;
    const Coef<R> k = load_coef<R>(sizeof(R) == 4 ? b.coef_f : b.coef_d, b.params, set, nz.dt);

    Slots<R, PPT> S;
    int64_t idx[PPT];
    bool act[PPT];
    // Thread t takes trajectories t, t + stride, ... of the tile.  A full tile has
    // stride kThreads; a partial one (the last tile of a set) ceil(count / PPT), so its
    // trajectories fill the slots of the first threads and whole warps beyond them stay
    // idle (their issue slots go to the SM's other blocks) instead of every thread
    // carrying one real and PPT - 1 empty slots through the paired instructions.  A
    // trajectory's arithmetic does not depend on its thread or slot: same results.
    const int stride = PPT > 1 ? (count + PPT - 1) / PPT : kThreads;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int li = lane_base + threadIdx.x + q * stride;
        act[q] = (int)threadIdx.x < stride && li < count;
        idx[q] = dchk(first + (act[q] ? li : count - 1), b.total_traj, b.dbg);
        S.y[q] = __ldcg(&s.y[idx[q]]);
        S.yacc[q] = __ldcg(&s.yacc[idx[q]]);
        S.ylo[q] = __ldcg(&s.ylo[idx[q]]);
        S.v[q] = __ldcg(&s.v[idx[q]]);
        S.e[q] = __ldcg(&s.e[idx[q]]);
        S.cell[q] = __ldcg(&s.cell[idx[q]]);
        if constexpr (sizeof(R) == 4) S.pb[q] = phase_base(S.y[q]);
        S.ss[q] = step_stream((uint64_t)idx[q] + nz.traj_base, K);
        if constexpr (MODE == kModeXorshift && !WS) {  // in a WS block the producer owns the generator
            const uint4 w = __ldcg(&st.xs[idx[q]]);
            S.xs[q][0] = w.x;
            S.xs[q][1] = w.y;
            S.xs[q][2] = w.z;
            S.xs[q][3] = w.w;
        }
    }

    const bool hist = h.bx > 0 || h.bv > 0;
    const R v_lo = (R)h.v_lo, v_hi = (R)h.v_hi;
    const R v_scale = h.bv > 0 ? (R)(h.bv / (h.v_hi - h.v_lo)) : (R)0;
    // Warps with no trajectory of the tile (a short tile) skip the stepping but
    // still reach the block's barriers.
    bool any_act = false;
#pragma unroll
    for (int q = 0; q < PPT; ++q) any_act |= act[q];
    const bool warp_live = __any_sync(0xffffffffu, any_act);

    if constexpr (WS) {
        wc->a0 = n_begin / kWsSlotSteps;
        wc->ready = 0;
    }
    int64_t n = n_begin;
    while (n < n_end) {
        int64_t seg_end = n_end;
        if (hist && h.snap_every > 0) seg_end = min(seg_end, (n / h.snap_every + 1) * h.snap_every);
        if (ck.every > 0) seg_end = min(seg_end, (n / ck.every + 1) * ck.every);
        if constexpr (WS) {
            if (warp_live) advance_ws<MODE == kModeHeun>(k, S, n, seg_end, *wc);
        } else {
            if (warp_live) advance<R, PPT, MODE, UNROLL>(k, K, S, n, seg_end);
        }
        n = seg_end;
        if (hist && (h.snap_every > 0 ? (n % h.snap_every == 0) : (n == N))) {
            const int64_t snap = dchk(h.snap_every > 0 ? n / h.snap_every - 1 : 0, h.n_snap, b.dbg);
            if constexpr (PACKED) {
                if (act[0]) {
                    const size_t row = (size_t)snap * b.n_sets + set;
                    if (h.bx > 0) atomicAdd(&h.x[row * h.bx + bin_x<R>(S.y[0] + S.yacc[0], h.bx)], 1u);
                    if (h.bv > 0)
                        atomicAdd(&h.v[row * (h.bv + 2) + bin_v<R>(S.v[0], v_lo, v_hi, v_scale, h.bv)], 1u);
                }
            } else {
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    if (!act[q]) continue;
                    if (h.bx > 0) atomicAdd(&sh[bin_x<R>(S.y[q] + S.yacc[q], h.bx)], 1u);
                    if (h.bv > 0) atomicAdd(&sh[h.bx + bin_v<R>(S.v[q], v_lo, v_hi, v_scale, h.bv)], 1u);
                }
                flush_hist<WS>(sh, h, snap, set, b.n_sets, 32);
            }
        }
        if (ck.every > 0 && n % ck.every == 0 && sizeof(R) == 4) {
            const int64_t slot = dchk(n / ck.every, ck.n_slots, b.dbg);
#pragma unroll
            for (int q = 0; q < PPT; ++q)
                if (act[q])
                    ck.ck[(size_t)slot * b.total_traj + idx[q]] =
                        make_float4((float)S.y[q], (float)S.yacc[q], (float)S.v[q], (float)S.e[q]);
        }
    }

#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        if (!act[q]) continue;
        s.y[idx[q]] = S.y[q];
        s.yacc[idx[q]] = S.yacc[q];
        s.ylo[idx[q]] = S.ylo[q];
        s.v[idx[q]] = S.v[q];
        s.e[idx[q]] = S.e[q];
        s.cell[idx[q]] = S.cell[q];
        if constexpr (MODE == kModeXorshift && !WS)
            st.xs[idx[q]] = make_uint4(S.xs[q][0], S.xs[q][1], S.xs[q][2], S.xs[q][3]);
    }
}

__device__ __forceinline__ void zero_hist(uint32_t *sh, const Hist &h) {
    if (h.bx > 0 || h.bv > 0) {
        const int nb = h.bx + (h.bv > 0 ? h.bv + 2 : 0);
        for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
}

// Lockstep schedule: one block per tile (narrow launch: `sub` blocks per tile,
// each taking blockDim.x consecutive trajectories of it), every tile over the
// window [g0, g1).
template <typename R, int PPT, bool PACKED, int MODE>
__global__ void ABP_INTEGRATE_BOUNDS integrate_kernel(Batch b, State st, Hist h, Ckpt ck, Noise nz,
                                                     KeyParam kp, int64_t g0, int64_t g1) {
    extern __shared__ uint32_t sh[];
    if constexpr (!PACKED) zero_hist(sh, h);
    const int sub = b.narrow ? (PACKED ? b.sub_packed : b.sub_single) : 1;
    const int tile = (PACKED ? b.n_single : 0) + (int)blockIdx.x / sub;
    const int lane_base = ((int)blockIdx.x % sub) * (int)blockDim.x;
    run_tile<R, PPT, PACKED, MODE, group_unroll<R, PPT, MODE, false>()>(b, st, h, ck, nz, kp.K, sh, tile, g0, g1,
                                                                       lane_base);
}

// Producer warp p of NP: the (nrs, trig) pairs of the launch's slots for the
// 32 trajectories of the consumer warp (lane by lane), in slot order, a slot
// rewritten only after the consumer handed it back.  The values are those
// single_step / group_step compute: same counter blocks (or, with xorshift
// noise, the same words of the trajectory's generator, which the first
// producer loads, advances over the launch's steps and stores back), same
// Box-Muller, same coefficient.
template <bool PACKED, int MODE, int NP>
__device__ __forceinline__ void ws_produce(const Batch &b, const State &st, const Noise &nz, const RoundKeys &K,
                                           const WsRing &r, int tile, int64_t w0, int64_t w1, int lane_base, int p) {
    constexpr int SS = kWsSlotSteps;
    const int64_t first = b.tile_first[tile];
    const int count = b.tile_count[tile];
    const int set_t = b.tile_set[tile];
    const int64_t N = b.set_steps[set_t];
    const int64_t n_begin = min(w0, N), n_end = min(w1, N);
    if (n_begin >= n_end) return;  // uniform over the block, as for the consumers
    if (MODE == kModeXorshift && p > 0) return;  // one generator chain per trajectory: the first producer's
    const int lane = threadIdx.x & 31;
    const int li = lane_base + lane;
    const bool act = li < count;
    const int64_t idx = dchk(first + (act ? li : count - 1), b.total_traj, b.dbg);
    if (!__any_sync(0xffffffffu, act)) return;  // the consumer warp does not step either
    if (tile == r.hold_tile) return;            // test hook: the consumer's waits run out
    const int set = PACKED ? packed_set(b, tile, min(li, count - 1)) : set_t;
    const Coef<float> k = load_coef<float>(b.coef_f, b.params, set, nz.dt);
    const StepStream ss = step_stream((uint64_t)idx + nz.traj_base, K);
    const int64_t a0 = n_begin / SS, a1 = (n_end - 1) / SS;
    bool failed = false;
    int32_t room = kWsSlots;  // slots of the launch [0, room) may be written
    uint32_t xs[4];
    if constexpr (MODE == kModeXorshift) {
        const uint4 w = __ldcg(&st.xs[idx]);
        xs[0] = w.x;
        xs[1] = w.y;
        xs[2] = w.z;
        xs[3] = w.w;
    }
    for (int64_t a = a0; a <= a1; ++a) {
        const int32_t kf = (int32_t)(a - a0);
        if (kf >= room) {
            const int32_t c = ws_wait(r.consumed, kf + 1 - kWsSlots, r, failed);
            room = failed ? INT32_MAX : c + kWsSlots;
        }
        float2 *out = r.buf + (size_t)(kf % kWsSlots) * SS * 32 + lane;
        if constexpr (MODE == kModeXorshift) {
            // the generator advances only over the launch's own steps (two words and the
            // Box-Muller cosine per step, as single_step draws them); a whole chunk of 16
            // steps takes its words first (the generator's serial chain), then the
            // transforms, independent of one another
            constexpr int CH = 16;
            const int64_t i0 = max(n_begin - a * SS, (int64_t)0), i1 = min(n_end - a * SS, (int64_t)SS);
            int64_t i = i0;
            for (; i + CH <= i1; i += CH) {
                uint32_t wv[2 * CH];
#pragma unroll
                for (int j = 0; j < 2 * CH; ++j) wv[j] = xorshift128(xs);
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    float nr, cs, sn;
                    box_muller_f32(wv[2 * j], wv[2 * j + 1], k.bm, nr, cs, sn);
                    out[(i + j) * 32] = make_float2(nr, cs);
                }
            }
            for (; i < i1; ++i) {
                const uint32_t wa = xorshift128(xs);
                const uint32_t wb = xorshift128(xs);
                float nr, cs, sn;
                box_muller_f32(wa, wb, k.bm, nr, cs, sn);
                out[i * 32] = make_float2(nr, cs);
            }
        } else {
            for (int j = p; j < SS / 4; j += NP) {
                const uint4 wv = step_block((uint32_t)(a * (SS / 4) + j), ss, K);
                float nr, cs, sn;
                box_muller_f32(wv.x, wv.y, k.bm, nr, cs, sn);
                out[(4 * j) * 32] = make_float2(nr, cs);
                out[(4 * j + 1) * 32] = make_float2(nr, sn);
                box_muller_f32(wv.z, wv.w, k.bm, nr, cs, sn);
                out[(4 * j + 2) * 32] = make_float2(nr, cs);
                out[(4 * j + 3) * 32] = make_float2(nr, sn);
            }
        }
        ws_publish(&r.filled[p], kf + 1);
    }
    if constexpr (MODE == kModeXorshift) {
        if (act) st.xs[idx] = make_uint4(xs[0], xs[1], xs[2], xs[3]);
    }
}

// Warp-specialised narrow lockstep launch (FP32, any scheme and noise): blocks
// of 32 (1 + NP) threads over the 32 trajectories a narrow block of 32 threads
// takes (sub blocks per tile); warp 0 steps them (run_tile), warps 1..NP
// produce their noise.  Dynamic shared memory: the histogram bins (one-set
// tiles), then the ring at the next 16-byte boundary.
template <bool PACKED, int MODE, int NP>
__global__ void __launch_bounds__(32 * (1 + NP)) ws_kernel(Batch b, State st, Hist h, Ckpt ck, Noise nz,
                                                          KeyParam kp, int64_t g0, int64_t g1, WaitCtl wait) {
    extern __shared__ uint32_t sh[];
    __shared__ int32_t filled[NP], consumed;
    if ((int)threadIdx.x < NP) filled[threadIdx.x] = 0;
    if (threadIdx.x == 0) consumed = 0;
    if constexpr (!PACKED) zero_hist(sh, h);
    __syncthreads();
    const int nb = PACKED ? 0 : h.bx + (h.bv > 0 ? h.bv + 2 : 0);
    float2 *ring = (float2 *)(sh + ((nb + 3) & ~3));
    if (smem_addr(ring) & 15) {  // uniform; never expected (dynamic shared memory is 16-byte aligned)
        if (threadIdx.x == 0) atomicCAS(wait.status, 0, 2);
        return;
    }
    const WsRing r{ring, filled, &consumed, wait.status, wait.limit_ns, wait.hold_tile};
    const int sub = PACKED ? b.sub_packed : b.sub_single;
    const int tile = (PACKED ? b.n_single : 0) + (int)blockIdx.x / sub;
    const int lane_base = ((int)blockIdx.x % sub) * 32;
    const int warp = (int)threadIdx.x >> 5;
    if (warp == 0) {
        WsCons c{r, MODE == kModeXorshift ? 1 : NP, 0, 0, false};
        run_tile<float, 1, PACKED, MODE, kGroupUnroll, true>(b, st, h, ck, nz, kp.K, sh, tile, g0, g1, lane_base, &c);
    } else {
        ws_produce<PACKED, MODE, NP>(b, st, nz, kp.K, r, tile, g0, g1, lane_base, warp - 1);
    }
}

__device__ __forceinline__ int load_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void store_release(int32_t *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Work-queue schedule: a persistent grid pops work items (tile, round) in a
// fixed order -- round-major, tiles of longer sets first -- where round j of
// a tile is its steps [g0 + j seg, g0 + (j+1) seg).  Round j of a tile may
// start only when round j-1 of that tile has been published; that item was
// popped earlier by a running block that itself waits only on items popped
// before it, so the earliest unfinished item is always runnable.  The wait is
// bounded: past q.wait_limit_ns the block records status 1 and every block
// leaves at its next check, without touching the item.
template <typename R, int PPT, int MODE>
__global__ void ABP_INTEGRATE_BOUNDS persistent_kernel(Batch b, State st, Hist h, Ckpt ck, Noise nz, KeyParam kp,
                                                      Queue q, int64_t g0, int64_t g1, int64_t seg) {
    extern __shared__ uint32_t sh[];
    __shared__ int s_tile, s_round;
    zero_hist(sh, h);
    for (;;) {
        if (threadIdx.x == 0) {
            int tile = -1, round = 0;
            const int item = atomicAdd(q.head, 1);
            if (item < q.n_items && *(volatile int32_t *)q.status == 0) {
                int lo = 0, hi = q.n_rounds - 1;  // last round whose start is <= item
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (q.round_start[mid] <= item)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                round = lo;
                tile = q.perm[item - q.round_start[round]];
                if (round > 0) {
                    const uint64_t t0 = global_ns();
                    while (load_acquire(&q.done[tile]) < round) {
                        if (*(volatile int32_t *)q.status != 0) {
                            tile = -1;
                            break;
                        }
                        if (global_ns() - t0 > (uint64_t)q.wait_limit_ns) {
                            atomicCAS(q.status, 0, 1);
                            tile = -1;
                            break;
                        }
                        __nanosleep(500);
                    }
                }
            }
            s_tile = tile;
            s_round = round;
        }
        __syncthreads();
        if (s_tile < 0) break;
        {
            const int64_t w0 = g0 + (int64_t)s_round * seg;
            run_tile<R, PPT, false, MODE, group_unroll<R, PPT, MODE, true>()>(b, st, h, ck, nz, kp.K, sh, s_tile, w0,
                                                                              min(w0 + seg, g1));
        }
        __syncthreads();  // every thread's state stores precede the publication
        if (threadIdx.x == 0 && s_tile != q.hold_tile) {
            __threadfence();
            store_release(&q.done[s_tile], s_round + 1);
        }
    }
}

// ---------------------------------------------------------------- reduction

// Fixed-order sum over the block of four doubles per thread; result valid in
// thread 0.
__device__ __forceinline__ void block_sum4(double (&a)[4], double (*red)[4]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] += __shfl_down_sync(0xffffffffu, a[j], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) red[warp][j] = a[j];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] = lane < nw ? red[lane][j] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int j = 0; j < 4; ++j) a[j] += __shfl_down_sync(0xffffffffu, a[j], o);
    }
}

// Adds the four terms of trajectory t to a.  Each square is rounded on its
// own before the addition (no fused multiply-add), as in a tree whose leaves
// are single trajectories.
template <typename R>
__device__ __forceinline__ void traj_terms(const SV<R> &s, int64_t t, double L, double inv_T, double (&a)[4]) {
    const double dx = L * disp_periods<R>(s, t);
    const double vbar = dx * inv_T;
    a[0] = __dadd_rn(a[0], vbar);
    a[1] = __dadd_rn(a[1], __dmul_rn(vbar, vbar));
    a[2] = __dadd_rn(a[2], dx);
    a[3] = __dadd_rn(a[3], __dmul_rn(dx, dx));
}

// Per tile: sum vbar, sum vbar^2, sum dx, sum dx^2 with dx = x_n - x_0 and
// vbar = dx / (n dt), n = min(g, N) steps done (the scheme advances x by
// v_k dt at every step, so dx / (n dt) is the time average of v_0 .. v_{n-1}).
template <typename R>
__global__ void __launch_bounds__(kThreads) tile_reduce_kernel(Batch b, State st, double dt, int64_t g,
                                                               double *partials) {
    __shared__ double red[kThreads / 32][4];
    const SV<R> s = view<R>(st);
    const int tile = blockIdx.x;
    const int set = (int)dchk(b.tile_set[tile], b.n_sets, b.dbg);
    const int64_t n = min(g, b.set_steps[set]);
    const double L = b.params[set].L;
    const double inv_T = n > 0 ? 1.0 / ((double)n * dt) : 0.0;
    const int64_t first = b.tile_first[tile];
    const int count = b.tile_count[tile];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int li = threadIdx.x; li < count; li += blockDim.x)
        traj_terms<R>(s, dchk(first + li, b.total_traj, b.dbg), L, inv_T, a);
    block_sum4(a, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) partials[(size_t)tile * 4 + j] = a[j];
}

// Sets of a combined ensemble: columns 0..3 of their moments rows recomputed from the
// sums in columns 4..7 (one thread per set; the sizes travel in the kernel arguments).
constexpr int kCombineChunk = 128;
struct CombineSizes {
    int64_t M[kCombineChunk], N[kCombineChunk];
};

__global__ void __launch_bounds__(kCombineChunk) combine_moments_kernel(double *moments, int32_t n, CombineSizes sz,
                                                                         double dt) {
    const int i = threadIdx.x;
    if (i >= n) return;
    double *row = moments + (size_t)i * 8;
    const double a[4] = {row[4], row[5], row[6], row[7]};
    moments_from_sums(row, a, sz.M[i], sz.N[i], dt);
}

// Per set in one-set tiles: fixed-order sum of its tiles' partials and the
// derived moments.  Block i takes set set_order[i] (or i).
template <typename R>
__global__ void __launch_bounds__(kThreads) set_reduce_kernel(Batch b, double dt, int64_t g, const double *partials,
                                                              double *moments) {
    __shared__ double red[kThreads / 32][4];
    const int set = b.set_order ? b.set_order[blockIdx.x] : (int)blockIdx.x;
    const int64_t n = min(g, b.set_steps[set]);
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t M = 0;
    const int t0 = b.set_tile_begin[set], t1 = b.set_tile_begin[set + 1];
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x)
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] += partials[(size_t)t * 4 + j];
    for (int t = t0; t < t1; ++t) M += b.tile_count[t];
    block_sum4(a, red);
    if (threadIdx.x == 0) moments_from_sums(moments + (size_t)set * 8, a, M, n, dt);
}

// Sets in packed tiles (fewer than kThreads trajectories each): one lane per
// set, 32 sets per warp, so the FP64 work of the moments (divisions, square
// root: slow on this GPU's FP64 pipe) is shared by 32 sets per instruction.
// A set must reduce to the same bits whether or not it was packed, i.e. in
// the order block_sum4 gives a one-tile set: a lane tree over each group of 32
// trajectories, then a lane tree over the groups' results.  For one or two
// trajectories that tree is the plain running sum (every other addition adds
// an exact zero), which the set's own lane does; larger sets are summed by the
// whole warp in the tree order, skipping the stages that only add zeros.
template <typename R>
__global__ void __launch_bounds__(kThreads) packed_reduce_kernel(Batch b, State st, double dt, int64_t g,
                                                                 double *moments) {
    const int n_packed = b.n_sets - b.n_unpacked;
    const int k = (int)(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    if ((k & ~31) >= n_packed) return;  // whole warps
    const int lane = threadIdx.x & 31;
    const bool mine = k < n_packed;
    const int set = mine ? (int)dchk(b.set_order[b.n_unpacked + k], b.n_sets, b.dbg) : 0;
    const SV<R> s = view<R>(st);
    const int64_t n = min(g, b.set_steps[set]);
    const double L = b.params[set].L;
    const double inv_T = n > 0 ? 1.0 / ((double)n * dt) : 0.0;
    const int64_t t0 = b.set_first[set], t1 = mine ? b.set_first[set + 1] : t0;
    const int m = (int)(t1 - t0);
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    if (m <= 2)
        for (int64_t t = t0; t < t1; ++t) traj_terms<R>(s, dchk(t, b.total_traj, b.dbg), L, inv_T, a);
    unsigned big = __ballot_sync(0xffffffffu, m > 2);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const int64_t u0 = __shfl_sync(0xffffffffu, t0, src);
        const int mu = __shfl_sync(0xffffffffu, m, src);
        const double Lu = __shfl_sync(0xffffffffu, L, src);
        const double iu = __shfl_sync(0xffffffffu, inv_T, src);
        const int groups = (mu + 31) >> 5;
        double part[4] = {0.0, 0.0, 0.0, 0.0};  // lane w: the tree sum of trajectories [32w, 32w + 32)
        for (int w = 0; w < groups; ++w) {
            double c[4] = {0.0, 0.0, 0.0, 0.0};
            if (w * 32 + lane < mu) traj_terms<R>(s, u0 + w * 32 + lane, Lu, iu, c);
            const int live = min(mu - w * 32, 32);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                if (o < live)
#pragma unroll
                    for (int j = 0; j < 4; ++j) c[j] += __shfl_down_sync(0xffffffffu, c[j], o);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double r = __shfl_sync(0xffffffffu, c[j], 0);
                if (lane == w) part[j] = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            if (o < groups)
#pragma unroll
                for (int j = 0; j < 4; ++j) part[j] += __shfl_down_sync(0xffffffffu, part[j], o);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double r = __shfl_sync(0xffffffffu, part[j], 0);
            if (lane == src) a[j] = r;
        }
    }
    if (mine) moments_from_sums(moments + (size_t)set * 8, a, m, n, dt);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) get_state_kernel(Batch b, State st, double dt, int64_t g, double *x,
                                                             double *x0, double *v, double *e, double *vbar) {
    const SV<R> s = view<R>(st);
    const int tile = blockIdx.x;
    const bool packed = tile >= b.n_single;
    const int64_t first = b.tile_first[tile];
    const int count = b.tile_count[tile];
    for (int li = threadIdx.x; li < count; li += blockDim.x) {
        const int64_t t = dchk(first + li, b.total_traj, b.dbg);
        const int set = packed ? packed_set(b, tile, li) : (int)dchk(b.tile_set[tile], b.n_sets, b.dbg);
        const int64_t n = min(g, b.set_steps[set]);
        const double L = b.params[set].L;
        const double x0t = L * (double)s.y0[t];
        const double dx = L * disp_periods<R>(s, t);
        if (x) x[t] = x0t + dx;
        if (x0) x0[t] = x0t;
        if (v) v[t] = (double)s.v[t];
        if (e) e[t] = (double)s.e[t];
        if (vbar) vbar[t] = n > 0 ? dx / ((double)n * dt) : 0.0;
    }
}

// ---------------------------------------------------------------- verification

__global__ void philox_kernel(uint32_t k0, uint32_t k1, const uint64_t *traj, const uint64_t *m, int64_t n,
                              uint32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 w = noise_block(m[i], traj[i], k0, k1);
        out[4 * i + 0] = w.x;
        out[4 * i + 1] = w.y;
        out[4 * i + 2] = w.z;
        out[4 * i + 3] = w.w;
    }
}

// The normals of the integrator's own noise path (step_block + box_muller_f32).
__global__ void normals_kernel(KeyParam kp, uint64_t traj, uint64_t n0, int64_t count, float *out) {
    const StepStream ss = step_stream(traj, kp.K);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t n = n0 + (uint64_t)i;
        const uint4 w = step_block((uint32_t)(n >> 2), ss, kp.K);
        out[i] = normal_from_block_f32(w, (uint32_t)(n & 3));
    }
}

size_t hist_smem(const Hist &h) { return sizeof(uint32_t) * (size_t)(h.bx + (h.bv > 0 ? h.bv + 2 : 0)); }

KeyParam key_param(uint32_t k0, uint32_t k1) {
    KeyParam kp;
    for (int r = 0; r < 10; ++r) {
        kp.K.rk[2 * r] = k0 + (uint32_t)r * kPhiloxW0;
        kp.K.rk[2 * r + 1] = k1 + (uint32_t)r * kPhiloxW1;
    }
    return kp;
}

template <typename R, int PPT, int MODE = kModeEM>
cudaError_t launch_persistent_t(const Batch &b, const State &s, const Hist &h, const Ckpt &c, const Noise &nz,
                                const Queue &q, int grid, int64_t g0, int64_t g1, int64_t seg, cudaStream_t st) {
    const size_t smem = hist_smem(h);
    auto kern = persistent_kernel<R, PPT, MODE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, kThreads, smem, st>>>(b, s, h, c, nz, key_param(nz.k0, nz.k1), q, g0, g1, seg);
    return cudaGetLastError();
}

// Raise the kernel's dynamic shared-memory limit to `smem` (the ring alone is
// 48 KB: with the static counters a block is past the default limit).
template <bool PACKED, int MODE>
cudaError_t ws_smem_limit(size_t smem) {
    return cudaFuncSetAttribute(ws_kernel<PACKED, MODE, kWsProducers>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

// Warp-specialised form of a narrow launch (see ws_kernel).
template <bool PACKED, int MODE>
cudaError_t launch_ws_t(const Batch &b, const State &s, const Hist &h, const Ckpt &c, const Noise &nz,
                        const KeyParam &kp, unsigned grid, size_t smem, int64_t g0, int64_t g1, const WaitCtl &wait,
                        cudaStream_t st) {
    const cudaError_t e = ws_smem_limit<PACKED, MODE>(smem);
    if (e != cudaSuccess) return e;
    ws_kernel<PACKED, MODE, kWsProducers><<<grid, 32 * (1 + kWsProducers), smem, st>>>(b, s, h, c, nz, kp, g0, g1,
                                                                                      wait);
    return cudaGetLastError();
}

// Whether `grid` blocks of the kernel fit on the GPU at once.
template <bool PACKED, int MODE>
cudaError_t ws_resident(unsigned grid, size_t smem, bool &fits) {
    auto kern = ws_kernel<PACKED, MODE, kWsProducers>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = ws_smem_limit<PACKED, MODE>(smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * (1 + kWsProducers), smem);
    fits = e == cudaSuccess && (int64_t)grid <= (int64_t)per_sm * sms;
    return e;
}

// Runs the launch warp-specialised (taken = true), unless the plan's width is over 32
// and the 32-thread stepping blocks would not all fit on the GPU at once.
template <int MODE>
cudaError_t launch_ws(const Batch &b0, const State &s, const Hist &h, const Ckpt &c, const Noise &nz, int64_t g0,
                      int64_t g1, const WaitCtl &wait, cudaStream_t st, bool &taken) {
    // 32 stepping threads per block whatever width w the plan chose (w divides the
    // tiles, so each of its blocks becomes w / 32 blocks): the tiles, and so every
    // result, stay the same
    Batch b = b0;
    b.sub_single = b0.sub_single * (b0.narrow / 32);
    b.sub_packed = b0.sub_packed * (b0.narrow / 32);
    const size_t ring = sizeof(float2) * (size_t)kWsSlots * kWsSlotSteps * 32;
    const size_t hist = (hist_smem(h) + 15) & ~(size_t)15;
    const unsigned grid_s = (unsigned)(b.n_single * b.sub_single);
    const unsigned grid_p = (unsigned)((b.n_tiles - b.n_single) * b.sub_packed);
    cudaError_t e = cudaSuccess;
    taken = true;
    if (b0.narrow > 32) {
        bool fits = true;
        if (grid_s > 0) e = ws_resident<false, MODE>(grid_s, hist + ring, fits);
        if (e == cudaSuccess && fits && grid_p > 0) e = ws_resident<true, MODE>(grid_p, ring, fits);
        if (e != cudaSuccess) return e;
        taken = fits;
        if (!fits) return cudaSuccess;
    }
    const KeyParam kp = key_param(nz.k0, nz.k1);
    if (grid_s > 0) e = launch_ws_t<false, MODE>(b, s, h, c, nz, kp, grid_s, hist + ring, g0, g1, wait, st);
    if (e == cudaSuccess && grid_p > 0) e = launch_ws_t<true, MODE>(b, s, h, c, nz, kp, grid_p, ring, g0, g1, wait, st);
    return e;
}

template <typename R, int PPT, int MODE = kModeEM>
cudaError_t launch_integrate_t(const Batch &b, const State &s, const Hist &h, const Ckpt &c, const Noise &nz,
                               int64_t g0, int64_t g1, cudaStream_t st, const WaitCtl *wait = nullptr) {
    const size_t smem = hist_smem(h);
    auto kern = integrate_kernel<R, PPT, false, MODE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if constexpr (sizeof(R) == 4 && PPT == 1 && ABP_WS) {
        if (b.narrow > 0 && b.narrow <= ABP_WS_WIDEST && wait && wait->status) {
            bool taken = false;
            const cudaError_t e = launch_ws<MODE>(b, s, h, c, nz, g0, g1, *wait, st, taken);
            if (e != cudaSuccess || taken) return e;
        }
    }
    const int threads = b.narrow ? b.narrow : kThreads;
    const int64_t sub_s = b.narrow ? b.sub_single : 1, sub_p = b.narrow ? b.sub_packed : 1;
    if (b.n_single > 0)
        kern<<<(unsigned)(b.n_single * sub_s), threads, smem, st>>>(b, s, h, c, nz, key_param(nz.k0, nz.k1), g0, g1);
    if (b.n_tiles > b.n_single)  // packed tiles: one trajectory per thread, histograms in global memory
        integrate_kernel<R, 1, true, MODE><<<(unsigned)((b.n_tiles - b.n_single) * sub_p), threads, 0, st>>>(
            b, s, h, c, nz, key_param(nz.k0, nz.k1), g0, g1);
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_init(const Batch &b, const State &s, const Hist &h, const Ckpt &c, const Noise &nz,
                        cudaStream_t st) {
    if (b.n_tiles == 0) return cudaSuccess;
    const size_t smem = hist_smem(h);
    if (s.fp64) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(init_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        init_kernel<double><<<b.n_tiles, kThreads, smem, st>>>(b, s, h, c, nz);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(init_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        init_kernel<float><<<b.n_tiles, kThreads, smem, st>>>(b, s, h, c, nz);
    }
    return cudaGetLastError();
}

cudaError_t launch_integrate(const Batch &b, const State &s, const Hist &h, const Ckpt &c, const Noise &nz, int ppt,
                             int64_t g0, int64_t g1, cudaStream_t st, const WaitCtl *wait) {
    if (b.n_tiles == 0 || g1 <= g0) return cudaSuccess;
    if (b.narrow) ppt = 1;
    if (s.fp64) {
        switch (ppt) {
            case 1: return launch_integrate_t<double, 1>(b, s, h, c, nz, g0, g1, st);
            case 2: return launch_integrate_t<double, 2>(b, s, h, c, nz, g0, g1, st);
            case 4: return launch_integrate_t<double, 4>(b, s, h, c, nz, g0, g1, st);
        }
    } else if (nz.scheme == 1) {
        switch (ppt) {
            case 1: return launch_integrate_t<float, 1, kModeHeun>(b, s, h, c, nz, g0, g1, st, wait);
            case 2: return launch_integrate_t<float, 2, kModeHeun>(b, s, h, c, nz, g0, g1, st);
            case 4: return launch_integrate_t<float, 4, kModeHeun>(b, s, h, c, nz, g0, g1, st);
        }
    } else if (nz.noise == 1) {
        switch (ppt) {
            case 1: return launch_integrate_t<float, 1, kModeXorshift>(b, s, h, c, nz, g0, g1, st, wait);
            case 2: return launch_integrate_t<float, 2, kModeXorshift>(b, s, h, c, nz, g0, g1, st);
            case 4: return launch_integrate_t<float, 4, kModeXorshift>(b, s, h, c, nz, g0, g1, st);
        }
    } else {
        switch (ppt) {
            case 1: return launch_integrate_t<float, 1>(b, s, h, c, nz, g0, g1, st, wait);
            case 2: return launch_integrate_t<float, 2>(b, s, h, c, nz, g0, g1, st);
            case 4: return launch_integrate_t<float, 4>(b, s, h, c, nz, g0, g1, st);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_persistent(const Batch &b, const State &s, const Hist &h, const Ckpt &c, const Noise &nz,
                              const Queue &q, int ppt, int grid, int64_t g0, int64_t g1, int64_t seg,
                              cudaStream_t st) {
    if (q.n_items == 0 || grid <= 0) return cudaSuccess;
    if (s.fp64) {
        switch (ppt) {
            case 1: return launch_persistent_t<double, 1>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
            case 2: return launch_persistent_t<double, 2>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
            case 4: return launch_persistent_t<double, 4>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
        }
    } else if (nz.scheme == 1) {
        switch (ppt) {
            case 1: return launch_persistent_t<float, 1, kModeHeun>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
            case 2: return launch_persistent_t<float, 2, kModeHeun>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
            case 4: return launch_persistent_t<float, 4, kModeHeun>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
        }
    } else if (nz.noise == 1) {
        switch (ppt) {
            case 1: return launch_persistent_t<float, 1, kModeXorshift>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
            case 2: return launch_persistent_t<float, 2, kModeXorshift>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
            case 4: return launch_persistent_t<float, 4, kModeXorshift>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
        }
    } else {
        switch (ppt) {
            case 1: return launch_persistent_t<float, 1>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
            case 2: return launch_persistent_t<float, 2>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
            case 4: return launch_persistent_t<float, 4>(b, s, h, c, nz, q, grid, g0, g1, seg, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename R, int MODE>
const void *persistent_fn(int ppt) {
    return ppt == 1 ? (const void *)persistent_kernel<R, 1, MODE>
           : ppt == 2 ? (const void *)persistent_kernel<R, 2, MODE> : (const void *)persistent_kernel<R, 4, MODE>;
}

cudaError_t persistent_occupancy(bool fp64, int ppt, size_t smem, int *blocks_per_sm, int mode) {
    const void *f = fp64 ? persistent_fn<double, kModeEM>(ppt)
                    : mode == kModeHeun ? persistent_fn<float, kModeHeun>(ppt)
                    : mode == kModeXorshift ? persistent_fn<float, kModeXorshift>(ppt)
                    : persistent_fn<float, kModeEM>(ppt);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kThreads, smem);
}

template <typename R, int MODE>
const void *integrate_fn(int ppt) {
    return ppt == 1 ? (const void *)integrate_kernel<R, 1, false, MODE>
           : ppt == 2 ? (const void *)integrate_kernel<R, 2, false, MODE> : (const void *)integrate_kernel<R, 4, false, MODE>;
}

cudaError_t integrate_occupancy(bool fp64, int ppt, size_t smem, int *blocks_per_sm, int mode) {
    const void *f = fp64 ? integrate_fn<double, kModeEM>(ppt)
                    : mode == kModeHeun ? integrate_fn<float, kModeHeun>(ppt)
                    : mode == kModeXorshift ? integrate_fn<float, kModeXorshift>(ppt)
                    : integrate_fn<float, kModeEM>(ppt);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kThreads, smem);
}

// One thread per set: its step coefficients in both state types (make_coef, the
// function every kernel would otherwise call at the start of each tile).
__global__ void coef_kernel(const abp_params *params, int32_t n, double dt, Coef<float> *cf, Coef<double> *cd) {
    const int i = (int)(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    if (i >= n) return;
    const abp_params p = params[i];
    cf[i] = make_coef<float>(p.q, p.c, p.d, p.gamma0, p.F0, p.D, p.h, p.L, p.asym, dt);
    cd[i] = make_coef<double>(p.q, p.c, p.d, p.gamma0, p.F0, p.D, p.h, p.L, p.asym, dt);
}

size_t coef_table_bytes(int32_t n_sets) {
    const size_t n = (size_t)std::max(n_sets, 1);
    return (sizeof(Coef<float>) * n + 255) / 256 * 256 + sizeof(Coef<double>) * n;
}

void coef_tables(void *buf, int32_t n_sets, const void **coef_f, const void **coef_d) {
    const size_t n = (size_t)std::max(n_sets, 1);
    *coef_f = buf;
    *coef_d = buf ? (const char *)buf + (sizeof(Coef<float>) * n + 255) / 256 * 256 : nullptr;
}

cudaError_t launch_coef(const abp_params *params, int32_t n_sets, double dt, void *buf, cudaStream_t st) {
    if (n_sets <= 0) return cudaSuccess;
    const void *cf, *cd;
    coef_tables(buf, n_sets, &cf, &cd);
    coef_kernel<<<(n_sets + kThreads - 1) / kThreads, kThreads, 0, st>>>(params, n_sets, dt, (Coef<float> *)cf,
                                                                         (Coef<double> *)cd);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const Batch &b, const State &s, const Noise &nz, int64_t g, double *partials,
                          double *moments, cudaStream_t st) {
    if (b.n_sets == 0) return cudaSuccess;
    if (b.n_single > 0) {
        if (s.fp64)
            tile_reduce_kernel<double><<<b.n_single, kThreads, 0, st>>>(b, s, nz.dt, g, partials);
        else
            tile_reduce_kernel<float><<<b.n_single, kThreads, 0, st>>>(b, s, nz.dt, g, partials);
    }
    if (b.n_unpacked > 0) {
        if (s.fp64)
            set_reduce_kernel<double><<<b.n_unpacked, kThreads, 0, st>>>(b, nz.dt, g, partials, moments);
        else
            set_reduce_kernel<float><<<b.n_unpacked, kThreads, 0, st>>>(b, nz.dt, g, partials, moments);
    }
    const int n_packed = b.n_sets - b.n_unpacked;
    if (n_packed > 0) {
        const int grid = (int)(((int64_t)n_packed + kThreads - 1) / kThreads);
        if (s.fp64)
            packed_reduce_kernel<double><<<grid, kThreads, 0, st>>>(b, s, nz.dt, g, moments);
        else
            packed_reduce_kernel<float><<<grid, kThreads, 0, st>>>(b, s, nz.dt, g, moments);
    }
    return cudaGetLastError();
}

cudaError_t launch_combine_moments(int32_t n, double *moments, const int64_t *M, const int64_t *N, double dt,
                                   cudaStream_t st) {
    for (int32_t i0 = 0; i0 < n; i0 += kCombineChunk) {
        const int32_t k = std::min<int32_t>(kCombineChunk, n - i0);
        CombineSizes sz;
        for (int32_t j = 0; j < kCombineChunk; ++j) {
            sz.M[j] = j < k ? M[i0 + j] : 0;
            sz.N[j] = j < k ? N[i0 + j] : 0;
        }
        combine_moments_kernel<<<1, kCombineChunk, 0, st>>>(moments + (size_t)i0 * 8, k, sz, dt);
    }
    return cudaGetLastError();
}

cudaError_t launch_get_state(const Batch &b, const State &s, double dt, int64_t g, double *x, double *x0, double *v,
                             double *e, double *vbar, cudaStream_t st) {
    if (b.n_tiles == 0) return cudaSuccess;
    if (s.fp64)
        get_state_kernel<double><<<b.n_tiles, kThreads, 0, st>>>(b, s, dt, g, x, x0, v, e, vbar);
    else
        get_state_kernel<float><<<b.n_tiles, kThreads, 0, st>>>(b, s, dt, g, x, x0, v, e, vbar);
    return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t k0, uint32_t k1, const uint64_t *traj, const uint64_t *m, int64_t n, uint32_t *out,
                          cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    philox_kernel<<<blocks, 256, 0, st>>>(k0, k1, traj, m, n, out);
    return cudaGetLastError();
}

cudaError_t launch_normals(uint32_t k0, uint32_t k1, uint64_t traj, uint64_t n0, int64_t count, float *out,
                           cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (n0 + (uint64_t)count > ((uint64_t)1 << 34)) return cudaErrorInvalidValue;  // step counters below 2^34
    const int blocks = (int)std::min<int64_t>((count + 255) / 256, 4096);
    normals_kernel<<<blocks, 256, 0, st>>>(key_param(k0, k1), traj, n0, count, out);
    return cudaGetLastError();
}

namespace {
// The first `count` words of one trajectory's xorshift stream (one thread: the
// stream is sequential by construction).
__global__ void xorshift_kernel(uint32_t k0, uint32_t k1, uint64_t traj, int64_t count, uint32_t *out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const uint4 w = xorshift_seed(traj, k0, k1);
    uint32_t s[4] = {w.x, w.y, w.z, w.w};
    for (int64_t i = 0; i < count; ++i) out[i] = xorshift128(s);
}
}  // namespace

cudaError_t launch_xorshift(uint32_t k0, uint32_t k1, uint64_t traj, int64_t count, uint32_t *out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    xorshift_kernel<<<1, 32, 0, st>>>(k0, k1, traj, count, out);
    return cudaGetLastError();
}

}  // namespace abp
