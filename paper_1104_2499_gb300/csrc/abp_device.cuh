// abp_device.cuh -- device building blocks of the ABP ensemble integrator
// (arXiv 1104.2499, Sec. 2 and Fig. 1): counter-based noise, Box-Muller, and one
// explicit Euler-Maruyama step of Eqs. (ereservoir), (velocity), (pot).
//
// State per trajectory: position x = L (cell + y + yacc + ylo) (see Coef
// below), velocity v, depot energy e.  The arithmetic type R is float
// (production) or double (precision-reference variant).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "abp.h"

namespace abp {

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Key (k0, k1), counter
// (c0..c3); 10 rounds, key bumped by the Weyl constants between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// One round.  The two products are written as 32 x 32 -> 64-bit multiplies, each
// a single wide integer multiply-add on the GPU (measured 5% faster integrator
// than separate high and low products).
__device__ __forceinline__ void philox_round(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0,
                                             uint32_t k1) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
    c0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    c1 = (uint32_t)p1;
    c2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c3 = (uint32_t)p0;
}

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(c0, c1, c2, c3, k0, k1);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Counter block m of trajectory t under seed (k0, k1).
__device__ __forceinline__ uint4 noise_block(uint64_t m, uint64_t t, uint32_t k0, uint32_t k1) {
    return philox4x32_10((uint32_t)m, (uint32_t)(m >> 32), (uint32_t)t, (uint32_t)(t >> 32), k0, k1);
}

// Round keys of a seed: rk[2r], rk[2r+1] = key of round r.  Passed to the
// integrator as a kernel parameter, so each key is an operand of the XOR.
struct RoundKeys {
    uint32_t rk[20];
};

// The step noise of one trajectory: counter (m, 0, t_lo, t_hi) for m < 2^32.
// The first round's products with the trajectory words do not depend on m
// and are formed once per trajectory (pre0 = hi(M1 t_lo) ^ k0, pre1 = lo(M1 t_lo)).
struct StepStream {
    uint32_t pre0, pre1, c3x;  // c3x = t_hi ^ k1 of round 0
};

__device__ __forceinline__ StepStream step_stream(uint64_t t, const RoundKeys &K) {
    StepStream s;
    const uint32_t tlo = (uint32_t)t, thi = (uint32_t)(t >> 32);
    const uint64_t p1 = (uint64_t)kPhiloxM1 * tlo;
    s.pre0 = (uint32_t)(p1 >> 32) ^ K.rk[0];  // c1 = m_hi = 0
    s.pre1 = (uint32_t)p1;
    s.c3x = thi ^ K.rk[1];
    return s;
}

#ifndef ABP_KEYS_IN_KERNEL
#define ABP_KEYS_IN_KERNEL 0
#endif

__device__ __forceinline__ uint4 step_block(uint32_t m, const StepStream &s, const RoundKeys &K) {
    // round 0 with the trajectory half precomputed
    const uint64_t p0 = (uint64_t)kPhiloxM0 * m;
    uint32_t c0 = s.pre0, c1 = s.pre1;
    uint32_t c2 = (uint32_t)(p0 >> 32) ^ s.c3x;
    uint32_t c3 = (uint32_t)p0;
#if ABP_KEYS_IN_KERNEL
    uint32_t k0 = K.rk[0], k1 = K.rk[1];
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
        philox_round(c0, c1, c2, c3, k0, k1);
    }
#else
#pragma unroll
    for (int r = 1; r < 10; ++r) philox_round(c0, c1, c2, c3, K.rk[2 * r], K.rk[2 * r + 1]);
#endif
    return make_uint4(c0, c1, c2, c3);
}

// Counter of the initial-condition draw (m = 2^63; step counters stay below 2^32).
constexpr uint64_t kInitCounter = 0x8000000000000000ull;
// Counter of the Philox block that seeds a trajectory's xorshift state.
constexpr uint64_t kXorshiftSeedCounter = kInitCounter + 1;

// Marsaglia's xorshift with four 32-bit words of state and shifts (11, 8, 19)
// (Xorshift RNGs, 2003), the generator of Fig. 1: (x, y, z, w) -> (y, z, w,
// w ^ (w >> 19) ^ t ^ (t >> 8)), t = x ^ (x << 11); returns the new w.
__device__ __forceinline__ uint32_t xorshift128(uint32_t (&s)[4]) {
    const uint32_t t = s[0] ^ (s[0] << 11);
    s[0] = s[1];
    s[1] = s[2];
    s[2] = s[3];
    s[3] = s[3] ^ (s[3] >> 19) ^ t ^ (t >> 8);
    return s[3];
}

// The xorshift state of global trajectory t: the Philox block of counter
// 2^63 + 1; an all-zero block (never met in practice) becomes (0, 0, 0, 1).
__device__ __forceinline__ uint4 xorshift_seed(uint64_t t, uint32_t k0, uint32_t k1) {
    uint4 w = noise_block(kXorshiftSeedCounter, t, k0, k1);
    if ((w.x | w.y | w.z | w.w) == 0u) w.w = 1u;
    return w;
}

// --------------------------------------------------------------------------
// Hardware approximations used by the FP32 path.  The approximate square
// root is the PTX instruction itself; log2 and sin/cos are CUDA's intrinsics.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

#ifndef ABP_ANGLE_FFMA
#define ABP_ANGLE_FFMA 1
#endif

constexpr double kPi = 3.14159265358979323846;
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kLn2F = 0.69314718055994530942f;

// Box-Muller of one word pair, FP32.  u1 = (wa + 1/2) 2^-32 (I2F rounds to
// nearest, the fused multiply-add adds the half exactly), u2 = floor(wb/2^9)
// 2^-23 built from the top 23 bits as f = 1 + u2 in [1, 2).  The angle is
// taken as 2 pi (u2 - 1/2) = 2 pi f - 3 pi in [-pi, pi), so the hardware
// sin/cos see a small argument; that flips both signs, which is folded into
// the returned (scaled) radius.  With c2 = -2 ln(2) s^2 for a scale s >= 0:
//   s z_even = nrs * cs,  s z_odd = nrs * sn,  nrs = -s sqrt(-2 ln u1).
__device__ __forceinline__ void box_muller_f32(uint32_t wa, uint32_t wb, float c2, float &nrs, float &cs,
                                               float &sn) {
    const float u1 = fmaf(__uint2float_rn(wa), 0x1p-32f, 0x1p-33f);
    const float l2 = __log2f(u1);  // <= 0
    nrs = -sqrt_approx(fabsf(l2 * c2));
    const float f = __uint_as_float(0x3f800000u | (wb >> 9));
#if ABP_ANGLE_FFMA
    __sincosf(fmaf(f, kTwoPiF, -1.5f * kTwoPiF), &sn, &cs);
#else
    __sincosf((f - 1.5f) * kTwoPiF, &sn, &cs);
#endif
}

// c2 of box_muller_f32 for the unscaled normal (s = 1).
constexpr float kBoxMullerUnit = -2.0f * kLn2F;

// Same mapping in FP64 (precision-reference variant).
__device__ __forceinline__ void box_muller_f64(uint32_t wa, uint32_t wb, double &z_even, double &z_odd) {
    const double u1 = ((double)wa + 0.5) * 0x1p-32;
    const double u2 = (double)(wb >> 9) * 0x1p-23;
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z_even = r * c;
    z_odd = r * s;
}

// --------------------------------------------------------------------------
// Per-set coefficients of the Euler-Maruyama map, built once per thread from
// the set's parameters.  With K = dt h 0.453 (2 pi / L) and c = cos phi,
//   -U'(x) dt = K (c + 2a cos 2phi) = K c + 4 a K c^2 - 2 a K      (Eq. (pot))
//   e' = e (1 - dt c - dt d v^2) + dt q                            (Eq. (ereservoir))
//   v' = v + [dt (d e - gamma0) v + dt F0 - 2aK + c (K + 4aK c) + sqrt(2 D dt) z]
//                                                                  (Eq. (velocity))
// The bracket (the increment) is formed first and added to v once.  Folding it
// into v (1 - dt gamma0 + dt d e) instead rounds that factor to a float near 1
// every step; its rounding error keeps its sign while e changes slowly, which
// acts as a friction error of ~1e-5 per unit time and, in FP32, used up most
// of the 1e-4 per-trajectory accuracy in 10^3 steps.
//   x' = x + v dt                                                  (dx/dt = v)
// Position.  x = L (cell + y + yacc + ylo): y is the fraction of the period,
// yacc collects the increments v dt / L of the current block of kBlockSteps
// steps (a small number, so each increment keeps almost all its bits), and
// at the block end yacc is added to y, whole periods move into cell and the
// rounding errors of both operations go to ylo, which only the displacement
// (never the force) reads.  This answers the single-precision caveat of the
// paper's Sec. 2: tiny increments are not added straight onto large values.
template <typename R>
struct Coef {
    R A;     // 1 - dt c
    R Bd;    // dt d
    R Cq;    // dt q
    R G;     // 1 - dt gamma0
    R Gd;    // -dt gamma0
    R Cm;    // -dt c
    R sigma; // sqrt(2 D dt)
    R bm;    // -2 ln(2) sigma^2: Box-Muller constant of the scaled radius
    R F;     // dt F0 - 2 a K
    R K;     // dt h 0.453 2 pi / L
    R A4;    // 4 a K
    R dtL;   // dt / L
    R hdtL;  // dt / (2 L)
};

// Phase of the potential: phi = 2 pi (y + 0.1903) = 2 pi (y - 0.8097) + 2 pi.
// The second form keeps |phi| < 2 pi for the y + yacc values that occur.
constexpr double kPhase = 0.1903;
constexpr double kPhaseShifted = 0.1903 - 1.0;

template <typename R>
__device__ __forceinline__ Coef<R> make_coef(double q, double c, double d, double gamma0, double F0, double D,
                                             double h, double L, double a, double dt) {
    Coef<R> k;
    const double K = dt * h * 0.453 * (2.0 * kPi / L);
    k.A = (R)(1.0 - dt * c);
    k.Bd = (R)(dt * d);
    k.Cq = (R)(dt * q);
    k.G = (R)(1.0 - dt * gamma0);
    k.Gd = (R)(-dt * gamma0);
    k.Cm = (R)(-dt * c);
    k.sigma = (R)sqrt(2.0 * D * dt);
    k.bm = (R)(-2.0 * 0.69314718055994530942 * 2.0 * D * dt);
    k.F = (R)(dt * F0 - 2.0 * a * K);
    k.K = (R)K;
    k.A4 = (R)(4.0 * a * K);
    k.dtL = (R)(dt / L);
    k.hdtL = (R)(0.5 * dt / L);
    return k;
}

// Coefficients of set `set`: from the batch's table when it has one (formed by
// make_coef in coef_kernel, so the same bits), else formed here from the parameters.
template <typename R>
__device__ __forceinline__ Coef<R> load_coef(const void *table, const abp_params *params, int set, double dt) {
    if (table) return static_cast<const Coef<R> *>(table)[set];
    const abp_params p = params[set];
    return make_coef<R>(p.q, p.c, p.d, p.gamma0, p.F0, p.D, p.h, p.L, p.asym, dt);
}

__device__ __forceinline__ float cos_phase(float y) {
    return __cosf(fmaf(y, kTwoPiF, (float)(2.0 * kPi * kPhaseShifted)));
}
__device__ __forceinline__ double cos_phase(double y) { return cospi(2.0 * (y + kPhase)); }

// FP32 phase of the force at position fraction y + yacc.  The fraction y only
// changes at the folds, so the integrator keeps pb = phase_base(y) beside it
// and each step forms the phase with one FMA from pb and yacc.
__device__ __forceinline__ float phase_base(float y) {
    return fmaf(y, kTwoPiF, (float)(2.0 * kPi * kPhaseShifted));
}
__device__ __forceinline__ float phase_arg(float pb, float yacc) { return fmaf(yacc, kTwoPiF, pb); }

// One Euler-Maruyama step; every right-hand side uses the step-n values.
// `sz` is sigma * z_n.
template <typename R>
__device__ __forceinline__ void em_step(const Coef<R> &k, R sz, R y, R &yacc, R &v, R &e) {
    const R cphi = cos_phase(y + yacc);
    const R t1 = fma(-k.Bd, v * v, k.A);
    const R hv = fma(k.Bd, e, k.Gd);
    const R a1 = sz + k.F;
    const R a2 = fma(hv, v, a1);
    const R P = fma(k.A4, cphi, k.K);
    const R dv = fma(P, cphi, a2);
    yacc = fma(v, k.dtL, yacc);
    e = fma(e, t1, k.Cq);
    v = v + dv;
}

// FP32 form with sigma folded into the Box-Muller radius: a1 = (-sigma r) *
// trig + F is one FMA.  pb = phase_base(y).
__device__ __forceinline__ void em_step_f32(const Coef<float> &k, float nrs, float trig, float pb, float &yacc,
                                            float &v, float &e) {
    const float cphi = __cosf(phase_arg(pb, yacc));
    const float t1 = fmaf(-k.Bd, v * v, k.A);
    const float hv = fmaf(k.Bd, e, k.Gd);
    const float a1 = fmaf(nrs, trig, k.F);
    const float a2 = fmaf(hv, v, a1);
    const float P = fmaf(k.A4, cphi, k.K);
    const float dv = fmaf(P, cphi, a2);
    yacc = fmaf(v, k.dtL, yacc);
    e = fmaf(e, t1, k.Cq);
    v = v + dv;
}

// One stochastic Heun step, FP32 (predictor-corrector for additive noise;
// Kloeden & Platen 1992, Sec. 15.1), on the same sigma z_n = nrs * trig as
// the Euler-Maruyama step.  With the drift increments of step n
//   dv = dt (d e - gamma0) v + dt F0 - 2aK + c (K + 4aK c),  de = dt (q - c e - d e v^2)
// the predictor is (x + v dt, v + dv + sigma z, e + de); its increments dv~,
// de~ give v' = v + (dv + dv~)/2 + sigma z, e' = e + (de + de~)/2 and
// x' = x + (v + v~) dt / 2.  Increments are formed on their own and added to
// the state once, as in em_step_f32.
__device__ __forceinline__ void heun_step_f32(const Coef<float> &k, float nrs, float trig, float pb, float &yacc,
                                              float &v, float &e) {
    const float sz = __fmul_rn(nrs, trig);  // kept a product: the compiler may not fuse it into the sums below
    const float c0 = __cosf(phase_arg(pb, yacc));
    const float dv0 = fmaf(fmaf(k.A4, c0, k.K), c0, fmaf(fmaf(k.Bd, e, k.Gd), v, k.F));
    const float de0 = fmaf(e, fmaf(-k.Bd, v * v, k.Cm), k.Cq);
    const float vp = v + (dv0 + sz);
    const float ep = e + de0;
    const float c1 = __cosf(phase_arg(pb, fmaf(v, k.dtL, yacc)));
    const float dv1 = fmaf(fmaf(k.A4, c1, k.K), c1, fmaf(fmaf(k.Bd, ep, k.Gd), vp, k.F));
    const float de1 = fmaf(ep, fmaf(-k.Bd, vp * vp, k.Cm), k.Cq);
    yacc = fmaf(v + vp, k.hdtL, yacc);  // (v + v~) dt / (2 L); halving is exact
    v = v + fmaf(0.5f, dv0 + dv1, sz);
    e = fmaf(0.5f, de0 + de1, e);
}

// --------------------------------------------------------------------------
// Paired FP32 arithmetic.  sm_100-family GPUs have two-lane FP32 instructions
// (__ffma2_rn, __fadd2_rn, __fmul2_rn): one instruction applies the same
// operation to the two halves of a register pair, each half rounded exactly as
// the scalar fmaf / + / * would round it.  A thread that holds two
// trajectories steps them with these, so the FP32 part of a step takes half
// the issue slots; the results are bitwise those of the scalar functions
// above (tested: paired and unpaired launches give the same state).
#ifndef ABP_F32X2
#define ABP_F32X2 1
#endif

__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// The coefficients of Coef<float> that the paired step reads, duplicated into
// both halves of a pair.
struct Coef2 {
    float2 A, nBd, Bd, Cq, Gd, F, K, A4, dtL, bm, Cm, hdtL;
};

__device__ __forceinline__ Coef2 make_coef2(const Coef<float> &k) {
    Coef2 c;
    c.A = dup2(k.A);
    c.nBd = dup2(-k.Bd);
    c.Bd = dup2(k.Bd);
    c.Cq = dup2(k.Cq);
    c.Gd = dup2(k.Gd);
    c.F = dup2(k.F);
    c.K = dup2(k.K);
    c.A4 = dup2(k.A4);
    c.dtL = dup2(k.dtL);
    c.bm = dup2(k.bm);
    c.Cm = dup2(k.Cm);
    c.hdtL = dup2(k.hdtL);
    return c;
}

// box_muller_f32 of two word pairs (wa.x, wb.x) and (wa.y, wb.y), same
// operations in the same order.
// Its two halves: the scaled radius from wa, and (cos, sin) of the angle from wb.
__device__ __forceinline__ float2 bm_radius_f32x2(uint2 wa, float2 c2) {
    const float2 u1 =
        __ffma2_rn(make_float2(__uint2float_rn(wa.x), __uint2float_rn(wa.y)), dup2(0x1p-32f), dup2(0x1p-33f));
    const float2 p = __fmul2_rn(make_float2(__log2f(u1.x), __log2f(u1.y)), c2);
    return make_float2(-sqrt_approx(fabsf(p.x)), -sqrt_approx(fabsf(p.y)));
}

__device__ __forceinline__ void bm_angle_f32x2(uint2 wb, float2 &cs, float2 &sn) {
    const float2 f = make_float2(__uint_as_float(0x3f800000u | (wb.x >> 9)), __uint_as_float(0x3f800000u | (wb.y >> 9)));
    const float2 ang = __ffma2_rn(f, dup2(kTwoPiF), dup2(-1.5f * kTwoPiF));
    __sincosf(ang.x, &sn.x, &cs.x);
    __sincosf(ang.y, &sn.y, &cs.y);
}

__device__ __forceinline__ void box_muller_f32x2(uint2 wa, uint2 wb, float2 c2, float2 &nrs, float2 &cs,
                                                 float2 &sn) {
    nrs = bm_radius_f32x2(wa, c2);
    bm_angle_f32x2(wb, cs, sn);
}

// em_step_f32 of two trajectories, same operations in the same order.
__device__ __forceinline__ void em_step_f32x2(const Coef2 &k, float2 nrs, float2 trig, float2 pb, float2 &yacc,
                                              float2 &v, float2 &e) {
    const float2 ph = __ffma2_rn(yacc, dup2(kTwoPiF), pb);
    const float2 cphi = make_float2(__cosf(ph.x), __cosf(ph.y));
    const float2 t1 = __ffma2_rn(k.nBd, __fmul2_rn(v, v), k.A);
    const float2 hv = __ffma2_rn(k.Bd, e, k.Gd);
    const float2 a1 = __ffma2_rn(nrs, trig, k.F);
    const float2 a2 = __ffma2_rn(hv, v, a1);
    const float2 P = __ffma2_rn(k.A4, cphi, k.K);
    const float2 dv = __ffma2_rn(P, cphi, a2);
    yacc = __ffma2_rn(v, k.dtL, yacc);
    e = __ffma2_rn(e, t1, k.Cq);
    v = __fadd2_rn(v, dv);
}

// heun_step_f32 of two trajectories, same operations in the same order.
__device__ __forceinline__ void heun_step_f32x2(const Coef2 &k, float2 nrs, float2 trig, float2 pb, float2 &yacc,
                                                float2 &v, float2 &e) {
    const float2 sz = __fmul2_rn(nrs, trig);
    const float2 ph0 = __ffma2_rn(yacc, dup2(kTwoPiF), pb);
    const float2 c0 = make_float2(__cosf(ph0.x), __cosf(ph0.y));
    const float2 dv0 = __ffma2_rn(__ffma2_rn(k.A4, c0, k.K), c0, __ffma2_rn(__ffma2_rn(k.Bd, e, k.Gd), v, k.F));
    const float2 de0 = __ffma2_rn(e, __ffma2_rn(k.nBd, __fmul2_rn(v, v), k.Cm), k.Cq);
    const float2 vp = __fadd2_rn(v, __fadd2_rn(dv0, sz));
    const float2 ep = __fadd2_rn(e, de0);
    const float2 ph1 = __ffma2_rn(__ffma2_rn(v, k.dtL, yacc), dup2(kTwoPiF), pb);
    const float2 c1 = make_float2(__cosf(ph1.x), __cosf(ph1.y));
    const float2 dv1 = __ffma2_rn(__ffma2_rn(k.A4, c1, k.K), c1, __ffma2_rn(__ffma2_rn(k.Bd, ep, k.Gd), vp, k.F));
    const float2 de1 = __ffma2_rn(ep, __ffma2_rn(k.nBd, __fmul2_rn(vp, vp), k.Cm), k.Cq);
    yacc = __ffma2_rn(__fadd2_rn(v, vp), k.hdtL, yacc);
    v = __fadd2_rn(v, __ffma2_rn(dup2(0.5f), __fadd2_rn(dv0, dv1), sz));
    e = __ffma2_rn(dup2(0.5f), __fadd2_rn(de0, de1), e);
}

template <typename R>
__device__ __forceinline__ R floor_r(R x);
template <>
__device__ __forceinline__ float floor_r<float>(float x) { return floorf(x); }
template <>
__device__ __forceinline__ double floor_r<double>(double x) { return floor(x); }

// Error-free sum (Knuth's TwoSum): s + err == a + b exactly.
template <typename R>
__device__ __forceinline__ R two_sum(R a, R b, R &err) {
    const R s = a + b;
    const R bb = s - a;
    err = (a - (s - bb)) + (b - bb);
    return s;
}

// End of a block of kBlockSteps steps: fold yacc into y and move whole
// periods into cell.  y's new value depends on (y, yacc) only; the rounding
// errors are added to ylo.
template <typename R>
__device__ __forceinline__ void fold_position(R &y, R &yacc, R &ylo, int32_t &cell) {
    R e1, e2;
    const R s = two_sum(y, yacc, e1);
    const R fl = floor_r<R>(s);
    const R w = two_sum(s, -fl, e2);
    y = w;
    yacc = 0;
    ylo += e1 + e2;
    cell += (int32_t)fl;
}

// The standard normal for step n from its counter block (generic, one step).
__device__ __forceinline__ float normal_from_block_f32(uint4 w, uint32_t k) {
    float nr, cs, sn;
    if (k < 2)
        box_muller_f32(w.x, w.y, kBoxMullerUnit, nr, cs, sn);
    else
        box_muller_f32(w.z, w.w, kBoxMullerUnit, nr, cs, sn);
    return (k & 1) ? nr * sn : nr * cs;
}

__device__ __forceinline__ double normal_from_block_f64(uint4 w, uint32_t k) {
    double ze, zo;
    if (k < 2)
        box_muller_f64(w.x, w.y, ze, zo);
    else
        box_muller_f64(w.z, w.w, ze, zo);
    return (k & 1) ? zo : ze;
}

// --------------------------------------------------------------------------
// Device clock and ordered shared-memory accesses (bounded producer/consumer
// hand-over between the warps of a block).
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int32_t ld_acquire_cta(const int32_t *p) {
    int32_t v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_cta(int32_t *p, int32_t v) {
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

}  // namespace abp
