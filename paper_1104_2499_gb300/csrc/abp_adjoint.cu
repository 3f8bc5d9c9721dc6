// abp_adjoint.cu -- pathwise adjoint of the ensemble mean velocity (abp_backward).
//
// With the noise held fixed, the Euler-Maruyama map s_{n+1} = Phi(s_n, theta, z_n)
// of Eqs. (ereservoir), (velocity), (pot) (Sec. 2) is differentiated in reverse:
//   lambda_n = (dPhi/ds_n)^T lambda_{n+1} + dJ/ds_n,     g += (dPhi/dtheta)^T lambda_{n+1}
// for J_i = sum_{n<N} v_n of each trajectory (the time-averaged velocity times N),
// theta = (D, q, c, d, gamma0, a).  The states are recomputed, not stored:
//   level 0  checkpoints in HBM every K steps, written by the forward integrator;
//   level 1  the K-step segment is re-run from its checkpoint, leaving a
//            sub-checkpoint every kSub steps in context-owned scratch memory;
//   level 2  each kSub-step sub-chunk is re-run from its sub-checkpoint into
//            registers and swept in reverse.
// Every re-run repeats the forward arithmetic bit for bit (same Philox words,
// same Box-Muller, same FMA sequence, same position folds), so the adjoint sees
// exactly the trajectory the forward produced.  Gradient terms are summed in
// FP32 within a segment and in FP64 across segments and trajectories.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "abp.h"
#include "abp_ctx.cuh"
#include "abp_device.cuh"
#include "abp_internal.cuh"

namespace abp {
namespace {

#ifndef ABP_ADJ_SUB
#define ABP_ADJ_SUB 8
#endif
#ifndef ABP_ADJ_MIN_BLOCKS
#define ABP_ADJ_MIN_BLOCKS 2
#endif
#ifndef ABP_ADJ_REV_THREADS
#define ABP_ADJ_REV_THREADS 256
#endif
// Reverse sweep with two trajectories per thread in paired FP32 (1) or one (0),
// and the block size and minimum resident blocks of the paired reverse kernel.
// Measured on the full differentiation workload (1M x 1e5, K = 1,000),
// backward time: one trajectory per thread 318 ms; paired, 210 registers (two
// 128-thread blocks per SM) 313 ms; paired, capped at 168 registers for three
// blocks per SM (no spills) 304 ms; paired with 4-step sub-chunks 324 ms.
#ifndef ABP_ADJ_REV_PAIRS
#define ABP_ADJ_REV_PAIRS 1
#endif
#ifndef ABP_ADJ_REV_PAIR_THREADS
#define ABP_ADJ_REV_PAIR_THREADS 128
#endif
#ifndef ABP_ADJ_REV_PAIR_MIN_BLOCKS
#define ABP_ADJ_REV_PAIR_MIN_BLOCKS 3
#endif
constexpr int kRevPairThreads = ABP_ADJ_REV_PAIR_THREADS;
// Level 1 with two trajectories per thread in paired FP32 (1) or one (0).
#ifndef ABP_ADJ_L1_PAIRS
#define ABP_ADJ_L1_PAIRS 1
#endif
// Aligned whole chunks of the paired level 1 stepped in groups of this many per
// loop iteration (1: one chunk per iteration).
#ifndef ABP_ADJ_L1_GROUP
#define ABP_ADJ_L1_GROUP 4
#endif
// Threads per block of the register-heavy reverse kernel (a multiple of 32).
constexpr int kRevThreads = ABP_ADJ_REV_THREADS;
// Threads per block of the level-1 kernel: small blocks, so that one fits on
// an SM beside the reverse kernel's blocks and fills the issue slots they
// leave idle.
constexpr int kL1Threads = 128;
constexpr int kSub = ABP_ADJ_SUB;  // steps per register-resident sub-chunk (a multiple of 4)
static_assert(kSub % 4 == 0 && (kBlockSteps % kSub) == 0, "sub-chunks hold whole Philox blocks");

struct AdjArgs {
    Batch b;
    Ckpt ck;
    Noise nz;
    RoundKeys K;        // Philox round keys of the seed (constant bank)
    float4 *sub;        // [n_sub][total_traj] sub-checkpoints (scratch)
    int64_t n_sub;      // sub-checkpoint slots per segment
    uint4 *words;       // [block][n_blk][2][threads] noise hand-off of the segment (scratch), WORDS kernels only
    int64_t n_blk;      // Philox blocks per segment (checkpoint_every / 4)
    const double *w;    // [n_sets] dJ/dmean_v, NULL = 1
    double *partials;   // [n_tiles][6]
};

// Noise hand-off from level 1 to the reverse sweep.  Level 1 draws every
// Philox block of its segment anyway; with WORDS it also stores, per block, the
// scaled radii of its two Box-Muller pairs and their two angle words (16 B per
// four steps of a trajectory), and the reverse sweep's level-2 re-run takes them
// from there instead of drawing the block and forming the radii a second time
// (it still forms the angles' sine and cosine).  The reverse kernel holds all the
// registers its three blocks per SM can have, so the blocks are not loaded into
// registers ahead of use: each thread copies its own chunk's blocks into shared
// memory with cp.async, kStages - 1 chunks ahead, and reads them when the chunk
// runs.  The radii are the bits box_muller_f32x2 returned in level 1, and the
// angles are formed by the same code, so every state and gradient is the same
// bit for bit with or without the hand-off.
#ifndef ABP_ADJ_STAGES
#define ABP_ADJ_STAGES 3
#endif
constexpr int kStages = ABP_ADJ_STAGES;

__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src_gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Noise of the four steps 4m .. 4m+3 as the forward integrator consumes it:
// the pair (nrs, trig) of each step is exactly what it feeds its fused
// multiply-add, so re-runs reproduce the forward states bit for bit.
__device__ __forceinline__ void block_noise(const Coef<float> &k, const StepStream &ss, const RoundKeys &K,
                                            uint32_t m, float (&nrs)[4], float (&tr)[4]) {
    const uint4 w = step_block(m, ss, K);
    float a, c, s;
    box_muller_f32(w.x, w.y, k.bm, a, c, s);
    nrs[0] = a;
    tr[0] = c;
    nrs[1] = a;
    tr[1] = s;
    box_muller_f32(w.z, w.w, k.bm, a, c, s);
    nrs[2] = a;
    tr[2] = c;
    nrs[3] = a;
    tr[3] = s;
}

// The same noise one step at a time, for segments that do not start on a
// multiple of 8 steps (one Philox block kept for its four steps).
struct NoiseCursor {
    uint32_t m;
    bool valid;
    float nrs[4], tr[4];

    __device__ void at(const Coef<float> &k, const StepStream &ss, const RoundKeys &K, int64_t n, float &nrs_n,
                       float &tr_n) {
        const uint32_t mm = (uint32_t)(n >> 2);
        if (!valid || mm != m) {
            block_noise(k, ss, K, mm, nrs, tr);
            m = mm;
            valid = true;
        }
        const int j = (int)(n & 3);
        nrs_n = j == 0 ? nrs[0] : j == 1 ? nrs[1] : j == 2 ? nrs[2] : nrs[3];
        tr_n = j == 0 ? tr[0] : j == 1 ? tr[1] : j == 2 ? tr[2] : tr[3];
    }
};

// One forward step at absolute index n, including the position fold the
// integrator applies after every kBlockSteps-th step (y depends on y and
// yacc only; the fold's error term and the cell index are not needed here).
__device__ __forceinline__ void fold(float &y, float &yacc, float &pb) {
    float lo = 0.0f;
    int32_t cell = 0;
    fold_position<float>(y, yacc, lo, cell);
    pb = phase_base(y);
}

__device__ __forceinline__ void fwd(const Coef<float> &k, float nrs, float trig, int64_t n, float &y, float &yacc,
                                   float &pb, float &v, float &e) {
    em_step_f32(k, nrs, trig, pb, yacc, v, e);
    if (((n + 1) & (kBlockSteps - 1)) == 0) fold(y, yacc, pb);
}

// One reverse step at the pre-step state (force phase ph, v = vv, e = ee,
// sigma z = sz): parameter terms with lambda_{n+1}, then lambda_n = J^T
// lambda_{n+1} + dJ/ds_n with dJ/dv_n = 1.
__device__ __forceinline__ void reverse_step(const Coef<float> &k, float kx, float dtf, float ph, float vv, float ee,
                                             float sz, float &lx, float &lv, float &le, float (&acc)[6]) {
    float sphi, cphi;
    __sincosf(ph, &sphi, &cphi);
    acc[0] = fmaf(lv, sz, acc[0]);                              // D
    acc[1] += le;                                               // q
    acc[2] = fmaf(le, ee, acc[2]);                              // c
    acc[3] = fmaf(ee * vv, fmaf(-le, vv, lv), acc[3]);          // d
    acc[4] = fmaf(lv, vv, acc[4]);                              // gamma0
    acc[5] = fmaf(lv, fmaf(2.0f * cphi, cphi, -1.0f), acc[5]);  // a
    const float dvdx = kx * sphi * fmaf(2.0f * k.A4, cphi, k.K);
    const float dvdv = fmaf(k.Bd, ee, k.G);
    const float dedv = -2.0f * k.Bd * ee * vv;
    const float dvde = k.Bd * vv;
    const float dede = fmaf(-k.Bd, vv * vv, k.A);
    const float nlx = fmaf(dvdx, lv, lx);
    const float nlv = fmaf(dtf, lx, fmaf(dvdv, lv, fmaf(dedv, le, 1.0f)));
    const float nle = fmaf(dvde, lv, dede * le);
    lx = nlx;
    lv = nlv;
    le = nle;
}

__device__ __forceinline__ void block_sum6(double (&a)[6], double (*red)[6]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < 6; ++j) a[j] += __shfl_down_sync(0xffffffffu, a[j], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < 6; ++j) red[warp][j] = a[j];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int j = 0; j < 6; ++j) a[j] = lane < nw ? red[lane][j] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int j = 0; j < 6; ++j) a[j] += __shfl_down_sync(0xffffffffu, a[j], o);
    }
}

// Level 1 of segment [s0, s1) of one trajectory: re-run from its checkpoint
// (y, yacc, v, e) = c0, leaving the state at s0, s0 + kSub, ... in the
// sub-checkpoint scratch.  Segments that start on a multiple of kSub steps run
// in whole kSub-step chunks whose noise comes one Philox block per four steps
// (the forward's own path); others step one at a time.
__device__ __forceinline__ void level1_segment(const AdjArgs &a, const Coef<float> &k, const StepStream &ss,
                                               int64_t idx, int64_t s0, int64_t s1, float4 c0) {
    const int64_t T = a.b.total_traj;
    float y = c0.x, yacc = c0.y, v = c0.z, e = c0.w;
    float pb = phase_base(y);
    const int n_chunks = (int)((s1 - s0 + kSub - 1) / kSub);
    const bool aligned = (s0 & (kSub - 1)) == 0;
    NoiseCursor nc;
    nc.valid = false;
    nc.m = 0;
    for (int j = 0; j < n_chunks; ++j) {
        const int64_t n0 = s0 + (int64_t)j * kSub;
        a.sub[(size_t)dchk(j, a.n_sub, a.b.dbg) * T + idx] = make_float4(y, yacc, v, e);
        const int len = (int)(s1 - n0 < kSub ? s1 - n0 : kSub);
        if (aligned && len == kSub) {
#pragma unroll
            for (int b2 = 0; b2 < kSub / 4; ++b2) {
                float nrs[4], tr[4];
                block_noise(k, ss, a.K, (uint32_t)(n0 >> 2) + b2, nrs, tr);
#pragma unroll
                for (int i = 0; i < 4; ++i) em_step_f32(k, nrs[i], tr[i], pb, yacc, v, e);
            }
            if (((n0 + kSub) & (kBlockSteps - 1)) == 0) fold(y, yacc, pb);
        } else {
            for (int i = 0; i < len; ++i) {
                float nrs, tr;
                nc.at(k, ss, a.K, n0 + i, nrs, tr);
                fwd(k, nrs, tr, n0 + i, y, yacc, pb, v, e);
            }
        }
    }
}

// level1_segment for two trajectories (idx0, idx1) of one thread: whole
// aligned chunks step the pair with paired FP32 instructions (same operations
// as em_step_f32 / box_muller_f32 on each half, so the sub-checkpoints are the
// scalar ones bit for bit); other chunks step each trajectory on its own.
// store1: whether the second trajectory is real (else it duplicates the first
// one's neighbour and its sub-checkpoints are not written).
// One Philox block of the hand-off for the thread's two trajectories: the
// scaled Box-Muller radii of its two word pairs (nrA, nrB, as their bits) and
// the two angle words, (nrA, wb_A, nrB, wb_B).  The buffer is laid out by
// kernel block -- [block][block index mrel in the segment][trajectory 0 / 1]
// [thread], the level-1 and reverse kernels mapping blocks and threads to
// trajectories alike -- so that wp (the thread's slot of mrel 0) plus a
// constant reaches every block of a chunk.  Both halves are stored, also where
// the thread's second trajectory repeats its first.
template <bool WORDS>
__device__ __forceinline__ void store_words(const AdjArgs &a, uint4 *wp, int64_t mrel, uint4 w0, uint4 w1, float2 nrA,
                                            float2 nrB) {
    if (WORDS) {
        const int64_t r = dchk(mrel, a.n_blk, a.b.dbg) * (2 * kL1Threads);
        wp[r] = make_uint4(__float_as_uint(nrA.x), w0.y, __float_as_uint(nrB.x), w0.w);
        wp[r + kL1Threads] = make_uint4(__float_as_uint(nrA.y), w1.y, __float_as_uint(nrB.y), w1.w);
    }
}

template <bool WORDS>
__device__ __forceinline__ void level1_segment2(const AdjArgs &a, const Coef<float> &k, const StepStream (&ss)[2],
                                                const int64_t (&idx)[2], bool store1, int64_t s0, int64_t s1,
                                                float4 c0, float4 c1) {
    const int64_t T = a.b.total_traj;
    uint4 *const wp = WORDS ? a.words + (size_t)blockIdx.x * (size_t)a.n_blk * (2 * kL1Threads) + threadIdx.x : nullptr;
    float y[2] = {c0.x, c1.x}, yacc[2] = {c0.y, c1.y}, v[2] = {c0.z, c1.z}, e[2] = {c0.w, c1.w};
    float pb[2] = {phase_base(y[0]), phase_base(y[1])};
    const int n_chunks = (int)((s1 - s0 + kSub - 1) / kSub);
    const bool aligned = (s0 & (kSub - 1)) == 0;
    const Coef2 k2 = make_coef2(k);
    NoiseCursor nc[2];
    nc[0].valid = nc[1].valid = false;
    nc[0].m = nc[1].m = 0;
    int j = 0;
#if ABP_ADJ_L1_GROUP > 1
    // aligned whole chunks in groups of ABP_ADJ_L1_GROUP: one loop iteration per group
    if (aligned) {
        const int full = (int)((s1 - s0) / kSub);
        float2 Y = make_float2(yacc[0], yacc[1]), V = make_float2(v[0], v[1]), E = make_float2(e[0], e[1]);
        float2 PB = make_float2(pb[0], pb[1]);
        for (; j + ABP_ADJ_L1_GROUP <= full; j += ABP_ADJ_L1_GROUP) {
#pragma unroll
            for (int c = 0; c < ABP_ADJ_L1_GROUP; ++c) {
                const int jc = j + c;
                const int64_t n0 = s0 + (int64_t)jc * kSub;
                const size_t js = (size_t)dchk(jc, a.n_sub, a.b.dbg);
                a.sub[js * T + idx[0]] = make_float4(y[0], Y.x, V.x, E.x);
                if (store1) a.sub[js * T + idx[1]] = make_float4(y[1], Y.y, V.y, E.y);
#pragma unroll
                for (int b2 = 0; b2 < kSub / 4; ++b2) {
                    const uint32_t m = (uint32_t)(n0 >> 2) + b2;
                    const uint4 w0 = step_block(m, ss[0], a.K), w1 = step_block(m, ss[1], a.K);
                    float2 nrA, nrB, cs, sn;
                    box_muller_f32x2(make_uint2(w0.x, w1.x), make_uint2(w0.y, w1.y), k2.bm, nrA, cs, sn);
                    em_step_f32x2(k2, nrA, cs, PB, Y, V, E);
                    em_step_f32x2(k2, nrA, sn, PB, Y, V, E);
                    box_muller_f32x2(make_uint2(w0.z, w1.z), make_uint2(w0.w, w1.w), k2.bm, nrB, cs, sn);
                    em_step_f32x2(k2, nrB, cs, PB, Y, V, E);
                    em_step_f32x2(k2, nrB, sn, PB, Y, V, E);
                    store_words<WORDS>(a, wp, 2 * (int64_t)jc + b2, w0, w1, nrA, nrB);
                }
                if (((n0 + kSub) & (kBlockSteps - 1)) == 0) {
                    yacc[0] = Y.x;
                    yacc[1] = Y.y;
                    fold(y[0], yacc[0], pb[0]);
                    fold(y[1], yacc[1], pb[1]);
                    Y = make_float2(yacc[0], yacc[1]);
                    PB = make_float2(pb[0], pb[1]);
                }
            }
        }
        yacc[0] = Y.x;
        yacc[1] = Y.y;
        v[0] = V.x;
        v[1] = V.y;
        e[0] = E.x;
        e[1] = E.y;
    }
#endif
    for (; j < n_chunks; ++j) {
        const int64_t n0 = s0 + (int64_t)j * kSub;
        const size_t js = (size_t)dchk(j, a.n_sub, a.b.dbg);
        a.sub[js * T + idx[0]] = make_float4(y[0], yacc[0], v[0], e[0]);
        if (store1) a.sub[js * T + idx[1]] = make_float4(y[1], yacc[1], v[1], e[1]);
        const int len = (int)(s1 - n0 < kSub ? s1 - n0 : kSub);
        if (aligned && len == kSub) {
            float2 Y = make_float2(yacc[0], yacc[1]), V = make_float2(v[0], v[1]), E = make_float2(e[0], e[1]);
            const float2 PB = make_float2(pb[0], pb[1]);
#pragma unroll
            for (int b2 = 0; b2 < kSub / 4; ++b2) {
                const uint32_t m = (uint32_t)(n0 >> 2) + b2;
                const uint4 w0 = step_block(m, ss[0], a.K), w1 = step_block(m, ss[1], a.K);
                float2 nrA, nrB, cs, sn;
                box_muller_f32x2(make_uint2(w0.x, w1.x), make_uint2(w0.y, w1.y), k2.bm, nrA, cs, sn);
                em_step_f32x2(k2, nrA, cs, PB, Y, V, E);
                em_step_f32x2(k2, nrA, sn, PB, Y, V, E);
                box_muller_f32x2(make_uint2(w0.z, w1.z), make_uint2(w0.w, w1.w), k2.bm, nrB, cs, sn);
                em_step_f32x2(k2, nrB, cs, PB, Y, V, E);
                em_step_f32x2(k2, nrB, sn, PB, Y, V, E);
                store_words<WORDS>(a, wp, 2 * (int64_t)j + b2, w0, w1, nrA, nrB);
            }
            yacc[0] = Y.x;
            yacc[1] = Y.y;
            v[0] = V.x;
            v[1] = V.y;
            e[0] = E.x;
            e[1] = E.y;
            if (((n0 + kSub) & (kBlockSteps - 1)) == 0) {
                fold(y[0], yacc[0], pb[0]);
                fold(y[1], yacc[1], pb[1]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 2; ++q)
                for (int i = 0; i < len; ++i) {
                    float nrs, tr;
                    nc[q].at(k, ss[q], a.K, n0 + i, nrs, tr);
                    fwd(k, nrs, tr, n0 + i, y[q], yacc[q], pb[q], v[q], e[q]);
                }
        }
    }
}

// Level 2 and the reverse sweep of segment [s0, s1): its kSub-step chunks in
// reverse order, each re-run from its sub-checkpoint into registers and swept
// backwards.  Each chunk's sub-checkpoint is loaded one chunk ahead, so its
// memory latency overlaps the previous chunk's arithmetic.
__device__ __forceinline__ void reverse_chunks(const AdjArgs &a, const Coef<float> &k, const StepStream &ss, float kx,
                                               float dtf, int64_t idx, int64_t s0, int64_t s1, float &lx, float &lv,
                                               float &le, float (&acc)[6]) {
    const int64_t T = a.b.total_traj;
    const int n_chunks = (int)((s1 - s0 + kSub - 1) / kSub);
    const bool aligned = (s0 & (kSub - 1)) == 0;
    NoiseCursor nc;
    nc.valid = false;
    nc.m = 0;
    float4 c_next = a.sub[(size_t)dchk(n_chunks - 1, a.n_sub, a.b.dbg) * T + idx];
    for (int j = n_chunks - 1; j >= 0; --j) {
        const int64_t n0 = s0 + (int64_t)j * kSub;
        const int len = (int)(s1 - n0 < kSub ? s1 - n0 : kSub);
        const float4 cj = c_next;
        if (j > 0) c_next = a.sub[(size_t)dchk(j - 1, a.n_sub, a.b.dbg) * T + idx];
        float y = cj.x, yacc = cj.y, v = cj.z, e = cj.w;
        float pb = phase_base(y);
        float ys[kSub], vs[kSub], es[kSub], szs[kSub];  // ys: the force phase of each step
        if (aligned && len == kSub) {
            // no fold falls inside an aligned chunk (folds come after multiples of kBlockSteps)
#pragma unroll
            for (int b2 = 0; b2 < kSub / 4; ++b2) {
                float nrs[4], tr[4];
                block_noise(k, ss, a.K, (uint32_t)(n0 >> 2) + b2, nrs, tr);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int q = 4 * b2 + i;
                    ys[q] = phase_arg(pb, yacc);
                    vs[q] = v;
                    es[q] = e;
                    szs[q] = nrs[i] * tr[i];
                    em_step_f32(k, nrs[i], tr[i], pb, yacc, v, e);
                }
            }
#pragma unroll
            for (int i = kSub - 1; i >= 0; --i) reverse_step(k, kx, dtf, ys[i], vs[i], es[i], szs[i], lx, lv, le, acc);
        } else {
            nc.valid = false;
#pragma unroll
            for (int i = 0; i < kSub; ++i) {
                if (i < len) {
                    float nrs, tr;
                    nc.at(k, ss, a.K, n0 + i, nrs, tr);
                    ys[i] = phase_arg(pb, yacc);
                    vs[i] = v;
                    es[i] = e;
                    szs[i] = nrs * tr;
                    fwd(k, nrs, tr, n0 + i, y, yacc, pb, v, e);
                }
            }
#pragma unroll
            for (int i = kSub - 1; i >= 0; --i)
                if (i < len) reverse_step(k, kx, dtf, ys[i], vs[i], es[i], szs[i], lx, lv, le, acc);
        }
    }
}

// reverse_step of two trajectories in the halves of FP32 pairs, same
// operations in the same order as the scalar function (each half rounded as
// the scalar operation), so the gradient sums are the scalar kernel's bits.
struct RevCoef2 {
    float2 kx, dtf, twoA4, K, Bd, G, m2Bd, nBd, A, one, mone, two, neg;
};

__device__ __forceinline__ RevCoef2 make_rev_coef2(const Coef<float> &k, float kx, float dtf) {
    RevCoef2 c;
    c.kx = dup2(kx);
    c.dtf = dup2(dtf);
    c.twoA4 = dup2(2.0f * k.A4);
    c.K = dup2(k.K);
    c.Bd = dup2(k.Bd);
    c.G = dup2(k.G);
    c.m2Bd = dup2(-2.0f * k.Bd);
    c.nBd = dup2(-k.Bd);
    c.A = dup2(k.A);
    c.one = dup2(1.0f);
    c.mone = dup2(-1.0f);
    c.two = dup2(2.0f);
    c.neg = dup2(-1.0f);
    return c;
}

__device__ __forceinline__ void reverse_step_x2(const RevCoef2 &c, float2 ph, float2 vv, float2 ee, float2 sz,
                                                float2 &lx, float2 &lv, float2 &le, float2 (&acc)[6]) {
    float2 sphi, cphi;
    __sincosf(ph.x, &sphi.x, &cphi.x);
    __sincosf(ph.y, &sphi.y, &cphi.y);
    acc[0] = __ffma2_rn(lv, sz, acc[0]);
    acc[1] = __fadd2_rn(acc[1], le);
    acc[2] = __ffma2_rn(le, ee, acc[2]);
    acc[3] = __ffma2_rn(__fmul2_rn(ee, vv), __ffma2_rn(__fmul2_rn(le, c.neg), vv, lv), acc[3]);
    acc[4] = __ffma2_rn(lv, vv, acc[4]);
    acc[5] = __ffma2_rn(lv, __ffma2_rn(__fmul2_rn(c.two, cphi), cphi, c.mone), acc[5]);
    const float2 dvdx = __fmul2_rn(__fmul2_rn(c.kx, sphi), __ffma2_rn(c.twoA4, cphi, c.K));
    const float2 dvdv = __ffma2_rn(c.Bd, ee, c.G);
    const float2 dedv = __fmul2_rn(__fmul2_rn(c.m2Bd, ee), vv);
    const float2 dvde = __fmul2_rn(c.Bd, vv);
    const float2 dede = __ffma2_rn(c.nBd, __fmul2_rn(vv, vv), c.A);
    const float2 nlx = __ffma2_rn(dvdx, lv, lx);
    const float2 nlv = __ffma2_rn(c.dtf, lx, __ffma2_rn(dvdv, lv, __ffma2_rn(dedv, le, c.one)));
    const float2 nle = __ffma2_rn(dvde, lv, __fmul2_rn(dede, le));
    lx = nlx;
    lv = nlv;
    le = nle;
}

// reverse_chunks for two trajectories of one thread (idx[0], idx[1]): whole
// aligned chunks run the level-2 re-run and the reverse sweep on FP32 pairs;
// other chunks run each trajectory on its own with the scalar functions.
// Shared-memory stage of the hand-off: [kStages][kSub / 4 blocks][2 trajectories][thread].
typedef uint4 WordStage[kSub / 4][2][kRevPairThreads];

template <bool WORDS>
__device__ __forceinline__ void reverse_chunks2(const AdjArgs &a, const Coef<float> &k, const StepStream (&ss)[2],
                                                float kx, float dtf, const int64_t (&idx)[2], int64_t s0, int64_t s1,
                                                float2 &lx, float2 &lv, float2 &le, float2 (&acc)[6],
                                                WordStage *stage) {
    const int64_t T = a.b.total_traj;
    const int n_chunks = (int)((s1 - s0 + kSub - 1) / kSub);
    const bool aligned = (s0 & (kSub - 1)) == 0;
    const int full = aligned ? (int)((s1 - s0) / kSub) : 0;  // chunks 0 .. full - 1 are whole
    const Coef2 k2 = make_coef2(k);
    const RevCoef2 rc = make_rev_coef2(k, kx, dtf);
    // WORDS: copy whole chunk jj's blocks into stage[jj % kStages]; one commit group per
    // call, empty for chunks that are not whole, so that groups and chunks stay in step
    const uint4 *const wr =
        WORDS ? a.words + (size_t)blockIdx.x * (size_t)a.n_blk * (2 * kRevPairThreads) + threadIdx.x : nullptr;
    auto fetch = [&](int jj) {
        if (jj >= 0 && jj < full) {
            WordStage &st = stage[jj % kStages];
#pragma unroll
            for (int b2 = 0; b2 < kSub / 4; ++b2) {
                const int64_t r = dchk(2 * (int64_t)jj + b2, a.n_blk, a.b.dbg) * (2 * kRevPairThreads);
                cp_async16(&st[b2][0][threadIdx.x], wr + r);
                cp_async16(&st[b2][1][threadIdx.x], wr + r + kRevPairThreads);
            }
        }
        cp_async_commit();
    };
    if (WORDS)
#pragma unroll
        for (int i = 0; i < kStages - 1; ++i) fetch(n_chunks - 1 - i);
    const size_t jl = (size_t)dchk(n_chunks - 1, a.n_sub, a.b.dbg);
    float4 n0c = a.sub[jl * T + idx[0]], n1c = a.sub[jl * T + idx[1]];
    for (int j = n_chunks - 1; j >= 0; --j) {
        const int64_t n0 = s0 + (int64_t)j * kSub;
        const int len = (int)(s1 - n0 < kSub ? s1 - n0 : kSub);
        const float4 c0 = n0c, c1 = n1c;
        if (j > 0) {
            const size_t jp = (size_t)dchk(j - 1, a.n_sub, a.b.dbg);
            n0c = a.sub[jp * T + idx[0]];
            n1c = a.sub[jp * T + idx[1]];
        }
        if (WORDS) {
            fetch(j - (kStages - 1));
            cp_async_wait<kStages - 1>();  // this thread's copies of chunk j have landed
        }
        if (aligned && len == kSub) {
            float2 Y = make_float2(c0.y, c1.y), V = make_float2(c0.z, c1.z), E = make_float2(c0.w, c1.w);
            const float2 PB = make_float2(phase_base(c0.x), phase_base(c1.x));
            float2 ys[kSub], vs[kSub], es[kSub], szs[kSub];
#pragma unroll
            for (int b2 = 0; b2 < kSub / 4; ++b2) {
                float2 nr[2], tr[4];
                float2 cs, sn;
                if (WORDS) {
                    // the radii come as level 1 formed them; the angles are formed here
                    const uint4 w0 = stage[j % kStages][b2][0][threadIdx.x];
                    const uint4 w1 = stage[j % kStages][b2][1][threadIdx.x];
                    nr[0] = make_float2(__uint_as_float(w0.x), __uint_as_float(w1.x));
                    nr[1] = make_float2(__uint_as_float(w0.z), __uint_as_float(w1.z));
                    bm_angle_f32x2(make_uint2(w0.y, w1.y), cs, sn);
                    tr[0] = cs;
                    tr[1] = sn;
                    bm_angle_f32x2(make_uint2(w0.w, w1.w), cs, sn);
                    tr[2] = cs;
                    tr[3] = sn;
                } else {
                    const uint32_t m = (uint32_t)(n0 >> 2) + b2;
                    const uint4 w0 = step_block(m, ss[0], a.K), w1 = step_block(m, ss[1], a.K);
                    box_muller_f32x2(make_uint2(w0.x, w1.x), make_uint2(w0.y, w1.y), k2.bm, nr[0], cs, sn);
                    tr[0] = cs;
                    tr[1] = sn;
                    box_muller_f32x2(make_uint2(w0.z, w1.z), make_uint2(w0.w, w1.w), k2.bm, nr[1], cs, sn);
                    tr[2] = cs;
                    tr[3] = sn;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int q = 4 * b2 + i;
                    ys[q] = __ffma2_rn(Y, dup2(kTwoPiF), PB);
                    vs[q] = V;
                    es[q] = E;
                    szs[q] = __fmul2_rn(nr[i >> 1], tr[i]);
                    em_step_f32x2(k2, nr[i >> 1], tr[i], PB, Y, V, E);
                }
            }
#pragma unroll
            for (int i = kSub - 1; i >= 0; --i) reverse_step_x2(rc, ys[i], vs[i], es[i], szs[i], lx, lv, le, acc);
        } else {
            // scalar path, one trajectory after the other
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float4 cq = q ? c1 : c0;
                float y = cq.x, yacc = cq.y, v = cq.z, e = cq.w;
                float pb = phase_base(y);
                float lxq = q ? lx.y : lx.x, lvq = q ? lv.y : lv.x, leq = q ? le.y : le.x;
                float accq[6];
#pragma unroll
                for (int r = 0; r < 6; ++r) accq[r] = q ? acc[r].y : acc[r].x;
                NoiseCursor nc;
                nc.valid = false;
                nc.m = 0;
                float ysq[kSub], vsq[kSub], esq[kSub], szq[kSub];
#pragma unroll
                for (int i = 0; i < kSub; ++i) {
                    if (i < len) {
                        float nrs, tr;
                        nc.at(k, ss[q], a.K, n0 + i, nrs, tr);
                        ysq[i] = phase_arg(pb, yacc);
                        vsq[i] = v;
                        esq[i] = e;
                        szq[i] = nrs * tr;
                        fwd(k, nrs, tr, n0 + i, y, yacc, pb, v, e);
                    }
                }
#pragma unroll
                for (int i = kSub - 1; i >= 0; --i)
                    if (i < len) reverse_step(k, kx, dtf, ysq[i], vsq[i], esq[i], szq[i], lxq, lvq, leq, accq);
                if (q) {
                    lx.y = lxq;
                    lv.y = lvq;
                    le.y = leq;
#pragma unroll
                    for (int r = 0; r < 6; ++r) acc[r].y = accq[r];
                } else {
                    lx.x = lxq;
                    lv.x = lvq;
                    le.x = leq;
#pragma unroll
                    for (int r = 0; r < 6; ++r) acc[r].x = accq[r];
                }
            }
        }
    }
}

// One launch per segment index and level, segments in reverse order: level 1
// (a plain forward re-run, light on registers) for segment `seg` of every
// trajectory, then level 2 and the reverse sweep (register-heavy) for the same
// segment.  The level-1 launch of segment seg - 1 runs on a second stream
// while the reverse sweep of segment seg runs, into the other of two
// sub-checkpoint buffers.  Between launches each trajectory keeps its adjoint
// state lambda = (x, v, e) and its six gradient sums in global memory.
// Trajectories of sets shorter than seg K skip.
struct SegView {
    float4 *lam;  // [total_traj] (lambda_x, lambda_v, lambda_e, -)
    double *G;    // [6][total_traj] gradient sums
};

// Both per-segment kernels run `sub` blocks per tile, block j of a tile taking
// its trajectories [j blockDim, (j + 1) blockDim): one trajectory per thread.
__global__ void __launch_bounds__(kL1Threads) adjoint_level1_kernel(AdjArgs a, int64_t seg, int sub) {
    const Batch &b = a.b;
    const int tile = (int)blockIdx.x / sub;
    const int li = ((int)blockIdx.x % sub) * (int)blockDim.x + (int)threadIdx.x;
    const int set = b.tile_set[tile];
    const int64_t N = b.set_steps[set], K = a.ck.every, T = b.total_traj;
    const int64_t s0 = seg * K;
    if (s0 >= N) return;  // uniform over the block
    const int64_t s1 = min(s0 + K, N);
    const Coef<float> k = load_coef<float>(b.coef_f, b.params, set, a.nz.dt);  // the forward's own coefficients
    if (li >= b.tile_count[tile]) return;
    const int64_t idx = dchk(b.tile_first[tile] + li, T, b.dbg);
    const StepStream ss = step_stream((uint64_t)idx + a.nz.traj_base, a.K);
    level1_segment(a, k, ss, idx, s0, s1, a.ck.ck[(size_t)dchk(seg, a.ck.n_slots, b.dbg) * T + idx]);
}

// Level 1 with two trajectories per thread (trajectories li and li +
// blockDim.x of the block's 2 blockDim.x), `sub` blocks per tile.
template <bool WORDS>
__global__ void __launch_bounds__(kL1Threads) adjoint_level1_pair_kernel(AdjArgs a, int64_t seg, int sub) {
    const Batch &b = a.b;
    const int tile = (int)blockIdx.x / sub;
    const int li = ((int)blockIdx.x % sub) * 2 * (int)blockDim.x + (int)threadIdx.x;
    const int set = b.tile_set[tile];
    const int64_t N = b.set_steps[set], K = a.ck.every, T = b.total_traj;
    const int64_t s0 = seg * K;
    if (s0 >= N) return;  // uniform over the block
    const int64_t s1 = min(s0 + K, N);
    const int count = b.tile_count[tile];
    if (li >= count) return;
    const Coef<float> k = load_coef<float>(b.coef_f, b.params, set, a.nz.dt);  // the forward's own coefficients
    const bool second = li + (int)blockDim.x < count;
    const int64_t idx[2] = {dchk(b.tile_first[tile] + li, T, b.dbg),
                            dchk(b.tile_first[tile] + (second ? li + (int)blockDim.x : li), T, b.dbg)};
    const StepStream ss[2] = {step_stream((uint64_t)idx[0] + a.nz.traj_base, a.K),
                              step_stream((uint64_t)idx[1] + a.nz.traj_base, a.K)};
    const int64_t slot = dchk(seg, a.ck.n_slots, b.dbg);
    level1_segment2<WORDS>(a, k, ss, idx, second, s0, s1, a.ck.ck[(size_t)slot * T + idx[0]],
                           a.ck.ck[(size_t)slot * T + idx[1]]);
}

__global__ void __launch_bounds__(kRevThreads, ABP_ADJ_MIN_BLOCKS) adjoint_reverse_kernel(AdjArgs a, SegView sv,
                                                                                          int64_t seg, int sub,
                                                                                          int64_t window) {
    const Batch &b = a.b;
    const int tile = (int)blockIdx.x / sub;
    const int li = ((int)blockIdx.x % sub) * (int)blockDim.x + (int)threadIdx.x;
    const int set = b.tile_set[tile];
    const int64_t N = b.set_steps[set], K = a.ck.every, T = b.total_traj;
    const int64_t s0 = seg * K;
    if (s0 >= N) return;  // uniform over the block
    const int64_t s1 = min(s0 + K, N);
    const abp_params p = b.params[set];
    const Coef<float> k = load_coef<float>(b.coef_f, b.params, set, a.nz.dt);  // the forward's own coefficients
    const float dtf = (float)a.nz.dt;
    const float kx = (float)(-2.0 * kPi / p.L);  // d phi / dx with the sign of d cos / d phi
    if (li >= b.tile_count[tile]) return;
    const int64_t idx = dchk(b.tile_first[tile] + li, T, b.dbg);
    const StepStream ss = step_stream((uint64_t)idx + a.nz.traj_base, a.K);
    float4 l0 = sv.lam[idx];
    // windowed adjoint: the window ending at step (seg + 1) K starts from zero
    if (window > 0 && ((seg + 1) * K) % window == 0) l0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float lx = l0.x, lv = l0.y, le = l0.z;
    float acc[6] = {0, 0, 0, 0, 0, 0};
    reverse_chunks(a, k, ss, kx, dtf, idx, s0, s1, lx, lv, le, acc);
    sv.lam[idx] = make_float4(lx, lv, le, 0.0f);
#pragma unroll
    for (int q = 0; q < 6; ++q) sv.G[(size_t)q * T + idx] += (double)acc[q];
}

// The reverse kernel with two trajectories per thread (trajectories li and
// li + blockDim.x of the block's 2 blockDim.x), `sub` blocks per tile.
template <bool WORDS>
__global__ void __launch_bounds__(kRevPairThreads, ABP_ADJ_REV_PAIR_MIN_BLOCKS) adjoint_reverse_pair_kernel(AdjArgs a, SegView sv, int64_t seg,
                                                                               int sub, int64_t window) {
    __shared__ WordStage stage[WORDS ? kStages : 1];
    const Batch &b = a.b;
    const int tile = (int)blockIdx.x / sub;
    const int li = ((int)blockIdx.x % sub) * 2 * (int)blockDim.x + (int)threadIdx.x;
    const int set = b.tile_set[tile];
    const int64_t N = b.set_steps[set], K = a.ck.every, T = b.total_traj;
    const int64_t s0 = seg * K;
    if (s0 >= N) return;  // uniform over the block
    const int64_t s1 = min(s0 + K, N);
    const int count = b.tile_count[tile];
    if (li >= count) return;
    const abp_params p = b.params[set];
    const Coef<float> k = load_coef<float>(b.coef_f, b.params, set, a.nz.dt);  // the forward's own coefficients
    const float dtf = (float)a.nz.dt;
    const float kx = (float)(-2.0 * kPi / p.L);
    const bool second = li + (int)blockDim.x < count;
    const int64_t idx[2] = {dchk(b.tile_first[tile] + li, T, b.dbg),
                            dchk(b.tile_first[tile] + (second ? li + (int)blockDim.x : li), T, b.dbg)};
    const StepStream ss[2] = {step_stream((uint64_t)idx[0] + a.nz.traj_base, a.K),
                              step_stream((uint64_t)idx[1] + a.nz.traj_base, a.K)};
    float4 l0 = sv.lam[idx[0]], l1 = sv.lam[idx[1]];
    if (window > 0 && ((seg + 1) * K) % window == 0) l0 = l1 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float2 lx = make_float2(l0.x, l1.x), lv = make_float2(l0.y, l1.y), le = make_float2(l0.z, l1.z);
    float2 acc[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[q] = make_float2(0.0f, 0.0f);
    reverse_chunks2<WORDS>(a, k, ss, kx, dtf, idx, s0, s1, lx, lv, le, acc, stage);
    sv.lam[idx[0]] = make_float4(lx.x, lv.x, le.x, 0.0f);
#pragma unroll
    for (int q = 0; q < 6; ++q) sv.G[(size_t)q * T + idx[0]] += (double)acc[q].x;
    if (second) {
        sv.lam[idx[1]] = make_float4(lx.y, lv.y, le.y, 0.0f);
#pragma unroll
        for (int q = 0; q < 6; ++q) sv.G[(size_t)q * T + idx[1]] += (double)acc[q].y;
    }
}

// Per tile: the initial-condition term, the parameter scales and the caller's
// weights, summed in FP64 over the tile's trajectories.
__global__ void __launch_bounds__(kThreads) adjoint_final_kernel(AdjArgs a, SegView sv) {
    __shared__ double red[kThreads / 32][6];
    const Batch &b = a.b;
    const int tile = blockIdx.x;
    const int set = b.tile_set[tile];
    const int64_t N = b.set_steps[set], T = b.total_traj;
    const abp_params p = b.params[set];
    const double dt = a.nz.dt;
    const int64_t first = b.tile_first[tile];
    const int count = b.tile_count[tile];
    int64_t M = 0;
    for (int t = b.set_tile_begin[set]; t < b.set_tile_begin[set + 1]; ++t) M += b.tile_count[t];
    double gsum[6] = {0, 0, 0, 0, 0, 0};
    if (N > 0) {
        // dmean_v/dtheta = (1 / (M N)) dJ_i/dtheta, scaled by the caller's weight
        const double wgt = (a.w ? a.w[set] : 1.0) / ((double)M * (double)N);
        const double Kd = dt * p.h * 0.453 * (2.0 * kPi / p.L);
        for (int li = threadIdx.x; li < count; li += blockDim.x) {
            const int64_t idx = first + li;
            double G[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) G[q] = sv.G[(size_t)q * T + idx];
            // initial condition: v0 = sqrt(D) z depends on D
            if (a.nz.v0_mode == 1) G[0] += (double)sv.lam[idx].y * (double)a.ck.ck[idx].z;
            gsum[0] += wgt * (p.D > 0.0 ? G[0] / (2.0 * p.D) : NAN);
            gsum[1] += wgt * dt * G[1];
            gsum[2] += wgt * (-dt) * G[2];
            gsum[3] += wgt * dt * G[3];
            gsum[4] += wgt * (-dt) * G[4];
            gsum[5] += wgt * 2.0 * Kd * G[5];
        }
    }
    block_sum6(gsum, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < 6; ++j) a.partials[(size_t)tile * 6 + j] = gsum[j];
}

// Per trajectory: d vbar_i / d theta (no caller weight, not averaged), from the same
// sums as adjoint_final_kernel -- the initial-condition term and the parameter scales
// applied, divided by the set's step count.  out: [total_traj][6].
__global__ void __launch_bounds__(kThreads) adjoint_traj_kernel(AdjArgs a, SegView sv, double *out) {
    const Batch &b = a.b;
    const int tile = blockIdx.x;
    const int set = b.tile_set[tile];
    const int64_t N = b.set_steps[set], T = b.total_traj;
    const abp_params p = b.params[set];
    const double dt = a.nz.dt;
    const double Kd = dt * p.h * 0.453 * (2.0 * kPi / p.L);
    const double inv_N = N > 0 ? 1.0 / (double)N : 0.0;
    const int64_t first = b.tile_first[tile];
    const int count = b.tile_count[tile];
    for (int li = threadIdx.x; li < count; li += blockDim.x) {
        const int64_t idx = dchk(first + li, T, b.dbg);
        double G[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) G[q] = sv.G[(size_t)q * T + idx];
        if (a.nz.v0_mode == 1) G[0] += (double)sv.lam[idx].y * (double)a.ck.ck[idx].z;
        double *o = out + (size_t)idx * 6;
        if (N == 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q) o[q] = 0.0;
            continue;
        }
        o[0] = (p.D > 0.0 ? G[0] / (2.0 * p.D) : NAN) * inv_N;
        o[1] = dt * G[1] * inv_N;
        o[2] = -dt * G[2] * inv_N;
        o[3] = dt * G[3] * inv_N;
        o[4] = -dt * G[4] * inv_N;
        o[5] = 2.0 * Kd * G[5] * inv_N;
    }
}

__global__ void __launch_bounds__(kThreads) adjoint_set_kernel(Batch b, const double *partials, double *grad) {
    __shared__ double red[kThreads / 32][6];
    const int set = blockIdx.x;
    const int t0 = b.set_tile_begin[set], t1 = b.set_tile_begin[set + 1];
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x)
#pragma unroll
        for (int j = 0; j < 6; ++j) a[j] += partials[(size_t)t * 6 + j];
    block_sum6(a, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < 6; ++j) grad[(size_t)set * 6 + j] = a[j];
}

abp_status set_err(abp_ctx *ctx, abp_status st, const char *msg, cudaError_t e = cudaSuccess) {
    ctx->err = msg;
    if (e != cudaSuccess) {
        ctx->err += ": ";
        ctx->err += cudaGetErrorString(e);
    }
    return st;
}

// Scratch of abp_backward, one allocation: the two sub-checkpoint buffers, the
// tile partials, the set gradients, the weights, lambda, the per-trajectory sums
// and, last, the two Philox-block buffers of the hand-off (0 bytes without it).
// abp_backward_traj reads lambda and the sums of the last call at the same offsets.
struct AdjLayout {
    size_t sub1, sub, part, grad, w, lam, g, words1, words, need;
    size_t off_part, off_grad, off_w, off_lam, off_g, off_words;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Kernel blocks per tile of the paired level-1 and reverse kernels (tiles hold up
// to kThreads * ppt trajectories, a block two per thread).
int pair_blocks_per_tile(const abp_ctx *ctx, int threads) {
    const int cap = kThreads * std::max(ctx->ppt, 1);
    return (cap + 2 * threads - 1) / (2 * threads);
}

AdjLayout adj_layout(const abp_ctx *ctx, bool words) {
    AdjLayout L;
    const int64_t T = ctx->total_traj, Kc = ctx->cfg.checkpoint_every;
    const int64_t n_sub = (Kc + kSub - 1) / kSub;
    L.sub1 = sizeof(float4) * (size_t)n_sub * (size_t)T;
    L.sub = 2 * align256(L.sub1);  // two buffers, alternating by segment
    L.part = sizeof(double) * 6 * (size_t)std::max(ctx->n_tiles, 1);
    L.grad = sizeof(double) * 6 * (size_t)std::max(ctx->n_sets, 1);
    L.w = sizeof(double) * (size_t)std::max(ctx->n_sets, 1);
    L.lam = sizeof(float4) * (size_t)std::max<int64_t>(T, 1);
    L.g = sizeof(double) * 6 * (size_t)std::max<int64_t>(T, 1);
    const size_t blocks = (size_t)ctx->n_tiles * (size_t)pair_blocks_per_tile(ctx, kL1Threads);
    L.words1 = words ? sizeof(uint4) * blocks * (size_t)(Kc / 4) * 2 * kL1Threads : 0;
    L.words = 2 * align256(L.words1);
    L.off_part = align256(L.sub);
    L.off_grad = L.off_part + align256(L.part);
    L.off_w = L.off_grad + align256(L.grad);
    L.off_lam = L.off_w + align256(L.w);
    L.off_g = L.off_lam + align256(L.lam);
    L.off_words = L.off_g + align256(L.g);
    L.need = L.off_words + L.words;
    return L;
}

// Whether abp_backward hands the Philox blocks from level 1 to the reverse sweep:
// the paired kernels, segments of whole sub-chunks, and both buffers within the
// budget -- ABP_ADJ_HANDOFF_BYTES if set (0: never), else half the free device
// memory not already held by the scratch.
bool use_handoff(const abp_ctx *ctx) {
    // both kernels must map blocks and threads to trajectories alike
    if (!ABP_ADJ_L1_PAIRS || !ABP_ADJ_REV_PAIRS || kL1Threads != kRevPairThreads) return false;
    if (ctx->cfg.checkpoint_every % kSub != 0) return false;
    const size_t bytes = adj_layout(ctx, true).words;
    const char *env = getenv("ABP_ADJ_HANDOFF_BYTES");
    if (env && *env) return (double)bytes <= strtod(env, nullptr);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return bytes <= (free_b + ctx->d_adj.cap) / 2;
}

}  // namespace
}  // namespace abp

using namespace abp;

extern "C" abp_status abp_backward(abp_ctx *ctx, const double *dJ_dmean_v, double *grad) {
    return abp_backward_windowed(ctx, dJ_dmean_v, grad, 0);
}

extern "C" abp_status abp_backward_windowed(abp_ctx *ctx, const double *dJ_dmean_v, double *grad, int64_t window) {
    const NvtxRange nvtx("abp_backward");
    if (!ctx) return ABP_EINVAL;
    if (window < 0 || (window > 0 && (ctx->cfg.checkpoint_every <= 0 || window % ctx->cfg.checkpoint_every != 0)))
        return set_err(ctx, ABP_EINVAL, "abp_backward_windowed: window must be a multiple of checkpoint_every");
    if (!grad) return set_err(ctx, ABP_EINVAL, "abp_backward: grad is NULL");
    const PtrKind kg = ptr_kind(grad, ctx->device);
    if (kg == PtrKind::OtherDevice) return set_err(ctx, ABP_EINVAL, "abp_backward: grad on another GPU");
    if (!ctx->have_batch) return set_err(ctx, ABP_ESTATE, "abp_backward before abp_set_params");
    if (ctx->cfg.checkpoint_every <= 0)
        return set_err(ctx, ABP_ESTATE, "abp_backward needs checkpoint_every > 0 during abp_integrate");
    if (ctx->g < ctx->max_steps) return set_err(ctx, ABP_ESTATE, "abp_backward before the integration completed");
    if (!ctx->ckpt_complete)
        return set_err(ctx, ABP_ESTATE, "abp_backward after abp_load: the checkpoints do not cover the run from step 0");
    const int64_t n_sub = (ctx->cfg.checkpoint_every + kSub - 1) / kSub;
    bool words = use_handoff(ctx);
    AdjLayout L = adj_layout(ctx, words);
    DevBuf &sc = ctx->d_adj;
    if (!sc.p || sc.cap < L.need) {
        sc.release();
        cudaError_t e = cudaMalloc(&sc.p, L.need);
        if (e != cudaSuccess && words) {  // no room for the hand-off: draw the blocks twice instead
            cudaGetLastError();
            words = false;
            L = adj_layout(ctx, false);
            e = cudaMalloc(&sc.p, L.need);
        }
        if (e != cudaSuccess) {
            sc.p = nullptr;
            cudaGetLastError();
            return set_err(ctx, ABP_ENOMEM, "abp_backward: scratch allocation failed", e);
        }
        sc.cap = L.need;
    }
    sc.bytes = L.need;
    char *base = (char *)sc.p;
    float4 *sub[2] = {(float4 *)base, (float4 *)(base + align256(L.sub1))};
    uint4 *wbuf[2] = {(uint4 *)(base + L.off_words), (uint4 *)(base + L.off_words + align256(L.words1))};
    double *partials = (double *)(base + L.off_part);
    double *gdev = (double *)(base + L.off_grad);
    double *wdev = (double *)(base + L.off_w);
    const size_t lam_bytes = L.lam, g_bytes = L.g;
    SegView sv;
    sv.lam = (float4 *)(base + L.off_lam);
    sv.G = (double *)(base + L.off_g);
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaSuccess;
    const double *w = nullptr;
    if (dJ_dmean_v) {
        const PtrKind kw = ptr_kind(dJ_dmean_v, ctx->device);
        if (kw == PtrKind::OtherDevice) return set_err(ctx, ABP_EINVAL, "abp_backward: weights on another GPU");
        if (kw == PtrKind::Device) {
            w = dJ_dmean_v;
        } else {
            e = cudaMemcpyAsync(wdev, dJ_dmean_v, sizeof(double) * ctx->n_sets, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return set_err(ctx, ABP_ECUDA, "abp_backward: weight upload", e);
            w = wdev;
        }
    }
    if (ctx->n_sets == 0) return ABP_OK;
    if (ctx->n_tiles > 0) {
        AdjArgs a;
        a.b = ctx->batch();
        a.ck = ctx->ckpt();
        a.nz = ctx->noise();
        a.sub = sub[0];
        a.n_sub = n_sub;
        a.words = nullptr;
        a.n_blk = ctx->cfg.checkpoint_every / 4;
        a.w = w;
        a.partials = partials;
        for (int r = 0; r < 10; ++r) {
            a.K.rk[2 * r] = a.nz.k0 + (uint32_t)r * kPhiloxW0;
            a.K.rk[2 * r + 1] = a.nz.k1 + (uint32_t)r * kPhiloxW1;
        }
        e = cudaMemsetAsync(sv.lam, 0, lam_bytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(sv.G, 0, g_bytes, s);
        if (e != cudaSuccess) return set_err(ctx, ABP_ECUDA, "abp_backward: clear", e);
        if (!ctx->aux) {
            e = cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking);
            for (int i = 0; e == cudaSuccess && i < 5; ++i)
                e = cudaEventCreateWithFlags(&ctx->adj_ev[i], cudaEventDisableTiming);
            if (e != cudaSuccess) {
                ctx->release_streams();
                return set_err(ctx, ABP_ECUDA, "abp_backward: stream set-up", e);
            }
        }
        cudaStream_t s2 = ctx->aux;
        cudaEvent_t *l1_done = ctx->adj_ev, *rev_done = ctx->adj_ev + 2, start = ctx->adj_ev[4];
        const int64_t Kc = ctx->cfg.checkpoint_every;
        const int64_t n_seg = (ctx->max_steps + Kc - 1) / Kc;
        // level 1 of segment j writes buffer j % 2; it may start once the reverse
        // sweep of segment j + 2, the last reader of that buffer, has finished
        e = cudaEventRecord(start, s);  // the checkpoints of the forward are complete
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, start, 0);
        // blocks per tile: tiles hold up to kThreads * ppt trajectories
        const int cap = kThreads * std::max(ctx->ppt, 1);
        const int sub1 = ABP_ADJ_L1_PAIRS ? pair_blocks_per_tile(ctx, kL1Threads) : (cap + kL1Threads - 1) / kL1Threads;
        const int sub2 = ABP_ADJ_REV_PAIRS ? pair_blocks_per_tile(ctx, kRevPairThreads)
                                           : (cap + kRevThreads - 1) / kRevThreads;
        auto level1 = [&](int64_t j) {
            AdjArgs aj = a;
            aj.sub = sub[j & 1];
            const unsigned g1 = (unsigned)((int64_t)ctx->n_tiles * sub1);
            if (words) {
                aj.words = wbuf[j & 1];
                adjoint_level1_pair_kernel<true><<<g1, kL1Threads, 0, s2>>>(aj, j, sub1);
            } else if (ABP_ADJ_L1_PAIRS)
                adjoint_level1_pair_kernel<false><<<g1, kL1Threads, 0, s2>>>(aj, j, sub1);
            else
                adjoint_level1_kernel<<<(unsigned)((int64_t)ctx->n_tiles * sub1), kL1Threads, 0, s2>>>(aj, j, sub1);
            return cudaEventRecord(l1_done[j & 1], s2);
        };
        if (e == cudaSuccess && n_seg > 0) e = level1(n_seg - 1);
        for (int64_t seg = n_seg - 1; e == cudaSuccess && seg >= 0; --seg) {
            if (seg > 0) {
                if (seg + 1 < n_seg) e = cudaStreamWaitEvent(s2, rev_done[(seg + 1) & 1], 0);
                if (e == cudaSuccess) e = level1(seg - 1);
            }
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, l1_done[seg & 1], 0);
            AdjArgs as = a;
            as.sub = sub[seg & 1];
            const unsigned g2 = (unsigned)((int64_t)ctx->n_tiles * sub2);
            if (words) {
                as.words = wbuf[seg & 1];
                adjoint_reverse_pair_kernel<true><<<g2, kRevPairThreads, 0, s>>>(as, sv, seg, sub2, window);
            } else if (ABP_ADJ_REV_PAIRS)
                adjoint_reverse_pair_kernel<false><<<g2, kRevPairThreads, 0, s>>>(as, sv, seg, sub2, window);
            else
                adjoint_reverse_kernel<<<(unsigned)((int64_t)ctx->n_tiles * sub2), kRevThreads, 0, s>>>(as, sv, seg,
                                                                                                       sub2, window);
            if (e == cudaSuccess) e = cudaEventRecord(rev_done[seg & 1], s);
            ctx->launches += 2;
        }
        if (e != cudaSuccess) return set_err(ctx, ABP_ECUDA, "abp_backward: launch", e);
        adjoint_final_kernel<<<ctx->n_tiles, kThreads, 0, s>>>(a, sv);
        ctx->launches += 1;
    }
    adjoint_set_kernel<<<ctx->n_sets, kThreads, 0, s>>>(ctx->batch(), partials, gdev);
    ctx->launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(ctx, ABP_ECUDA, "abp_backward: launch", e);
    const size_t out_bytes = sizeof(double) * 6 * (size_t)ctx->n_sets;
    if (kg == PtrKind::Device) {
        e = cudaMemcpyAsync(grad, gdev, out_bytes, cudaMemcpyDeviceToDevice, s);
    } else {
        e = cudaMemcpyAsync(grad, gdev, out_bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return set_err(ctx, ABP_ECUDA, "abp_backward: gradient copy", e);
    ctx->adj_valid = true;
    return ABP_OK;
}

extern "C" abp_status abp_backward_traj(abp_ctx *ctx, double *dvbar) {
    const NvtxRange nvtx("abp_backward_traj");
    if (!ctx) return ABP_EINVAL;
    if (!dvbar) return set_err(ctx, ABP_EINVAL, "abp_backward_traj: dvbar is NULL");
    if (!ctx->have_batch || !ctx->adj_valid)
        return set_err(ctx, ABP_ESTATE, "abp_backward_traj: no abp_backward since the batch was last (re)started");
    const PtrKind k = ptr_kind(dvbar, ctx->device);
    if (k == PtrKind::OtherDevice) return set_err(ctx, ABP_EINVAL, "abp_backward_traj: output on another GPU");
    const int64_t T = ctx->total_traj;
    if (T == 0 || ctx->n_tiles == 0) return ABP_OK;
    // the per-trajectory sums of the last backward call: the same scratch layout as there
    const int64_t n_sub = (ctx->cfg.checkpoint_every + kSub - 1) / kSub;
    const AdjLayout L = adj_layout(ctx, false);  // the hand-off buffers come after the sums
    char *base = (char *)ctx->d_adj.p;
    SegView sv;
    sv.lam = (float4 *)(base + L.off_lam);
    sv.G = (double *)(base + L.off_g);
    AdjArgs a;
    a.b = ctx->batch();
    a.ck = ctx->ckpt();
    a.nz = ctx->noise();
    a.sub = nullptr;
    a.n_sub = n_sub;
    a.words = nullptr;
    a.n_blk = 0;
    a.w = nullptr;
    a.partials = nullptr;
    cudaStream_t s = ctx->stream;
    const size_t bytes = sizeof(double) * 6 * (size_t)T;
    DevBuf tmp;
    double *dst = dvbar;
    if (k != PtrKind::Device) {
        const cudaError_t ea = cudaMalloc(&tmp.p, bytes);
        if (ea != cudaSuccess) {
            tmp.p = nullptr;
            cudaGetLastError();
            return set_err(ctx, ABP_ENOMEM, "abp_backward_traj: staging buffer", ea);
        }
        dst = (double *)tmp.p;
    }
    adjoint_traj_kernel<<<ctx->n_tiles, kThreads, 0, s>>>(a, sv, dst);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && k != PtrKind::Device) {
        e = cudaMemcpyAsync(dvbar, dst, bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    tmp.release();
    if (e != cudaSuccess) return set_err(ctx, ABP_ECUDA, "abp_backward_traj", e);
    return ABP_OK;
}
