/*
 * abp_oracle.c -- plain, slow FP64 reference for the active-Brownian-particle
 * ensemble of arXiv 1104.2499 (Zabicki, "OpenCL/OpenGL approach for studying
 * active Brownian motion").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may include, link or
 * call this file: it is used by the tests, by the smoke check and by the
 * benchmark's CPU-baseline leg, and by nothing else.  It shares no code,
 * header, constant table or helper with the CUDA path; every piece below is
 * written from the paper's equations and from the published definition of
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11).
 *
 * What it computes, in the paper's notation (Sec. 2):
 *   Eq. (ereservoir)  de/dt = q - c e - d e v^2
 *   Eq. (velocity)    dv/dt = F0 + d e v - gamma v - U'(x) + sqrt(2D) xi(t)
 *   Eq. (pot)         U(x)  = h [0.499 - 0.453 (sin phi + a sin 2 phi)],
 *                     phi   = 2 pi (x/L + 0.1903)
 *   kinematics        dx/dt = v
 * integrated by explicit Euler-Maruyama (all right-hand sides taken at step n),
 * with the Gaussian noise of Fig. 1 (a Box-Muller transformation) drawn from a
 * counter-based Philox4x32-10 stream keyed by (seed, trajectory, step); or, as
 * a higher-order variant the paper does not use, by the stochastic Heun
 * predictor-corrector on the same noise (or_heun_step).
 *
 * Readings of the paper taken where it is silent or garbled:
 *   - the trailing "{v}" after xi(t) in Eq. (velocity) is a typesetting
 *     artefact: the noise is additive, sqrt(2D) xi;
 *   - the second harmonic of Eq. (pot) is sin(4 pi (x + 0.1903)) with weight
 *     a (a = 1/4 in the paper); with it U has its minimum exactly at x = 0;
 *   - the period L scales the argument as x/L;
 *   - gamma is a constant friction coefficient gamma0;
 *   - the uniform-variate mapping of Box-Muller is
 *       u1 = (w_a + 1/2) 2^-32           in (0, 1)
 *       u2 = floor(w_b / 2^9) 2^-23      in [0, 1)
 *     z_cos = sqrt(-2 ln u1) cos(2 pi u2) feeds the even step of a pair and
 *     z_sin = sqrt(-2 ln u1) sin(2 pi u2) the odd step;
 *   - Philox counter for step n of global trajectory id t under seed s:
 *       key = (s_lo, s_hi), ctr = (m_lo, m_hi, t_lo, t_hi), m = n >> 2,
 *     words (w0,w1) -> steps 4m, 4m+1 and (w2,w3) -> steps 4m+2, 4m+3;
 *     the initial condition uses m = 2^63 (ctr = (0, 0x80000000, t_lo, t_hi)):
 *       x0 = L floor(w0 / 2^8) 2^-24, v0 = 0 or sqrt(D) * z_cos(w1, w2), e0 = 0;
 *   - the time-averaged velocity of a trajectory is (1/N) sum_{n<N} v_n.
 *
 * Parity is pinned (tests/test_oracle_pins.py) against: ATen's host Philox
 * engine (independent implementation), closed forms of the free and
 * constant-force limits, the depot and active-motion fixed points, the
 * Boltzmann stationary density of the passive particle, symmetry of the
 * current at a = 0, and central finite differences for the tangent-linear
 * gradient.  The value of the ratchet current itself has no pin in the paper
 * (its Fig. 2 is not reproduced): parity unpinned for that number beyond the
 * statistical identities above.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 Philox S-box,
 * multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 /
 * 0xBB67AE85. */

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof(c));
}

/* The four words of counter m of trajectory `traj` under `seed`. */
void or_noise_words(uint64_t seed, uint64_t traj, uint64_t m, uint32_t out[4])
{
    const uint32_t ctr[4] = {(uint32_t)m, (uint32_t)(m >> 32), (uint32_t)traj,
                             (uint32_t)(traj >> 32)};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* Box-Muller transformation (Fig. 1) of one pair of words. */
void or_box_muller(uint32_t wa, uint32_t wb, double z[2])
{
    const double u1 = ((double)wa + 0.5) * 0x1p-32;
    const double u2 = (double)(wb >> 9) * 0x1p-23;
    const double r = sqrt(-2.0 * log(u1));
    z[0] = r * cos(2.0 * M_PI * u2);
    z[1] = r * sin(2.0 * M_PI * u2);
}

/* The standard normal z_n that drives step n of trajectory `traj`. */
double or_normal(uint64_t seed, uint64_t traj, uint64_t n)
{
    uint32_t w[4];
    double z[2];
    or_noise_words(seed, traj, n >> 2, w);
    const int k = (int)(n & 3u);
    if (k < 2)
        or_box_muller(w[0], w[1], z);
    else
        or_box_muller(w[2], w[3], z);
    return z[k & 1];
}

/* z_n for n = n0 .. n0 + count - 1 of one trajectory (bulk form of or_normal). */
void or_normals(uint64_t seed, uint64_t traj, uint64_t n0, int64_t count, double *out)
{
    for (int64_t i = 0; i < count; ++i)
        out[i] = or_normal(seed, traj, n0 + (uint64_t)i);
}

/* ------------------------------------------------------------------------ */
/* Model (Sec. 2). */

typedef struct {
    double q, c, d, gamma0, F0, D, h, L, asym;
} or_params;

static double phase(const or_params *p, double x) { return 2.0 * M_PI * (x / p->L + 0.1903); }

/* Eq. (pot). */
double or_potential(const or_params *p, double x)
{
    const double ph = phase(p, x);
    return p->h * (0.499 - 0.453 * (sin(ph) + p->asym * sin(2.0 * ph)));
}

/* dU/dx. */
double or_potential_dx(const or_params *p, double x)
{
    const double ph = phase(p, x);
    const double k = 2.0 * M_PI / p->L;
    return -p->h * 0.453 * k * (cos(ph) + 2.0 * p->asym * cos(2.0 * ph));
}

/* d2U/dx2 (tangent-linear only). */
static double potential_dxx(const or_params *p, double x)
{
    const double ph = phase(p, x);
    const double k = 2.0 * M_PI / p->L;
    return p->h * 0.453 * k * k * (sin(ph) + 4.0 * p->asym * sin(2.0 * ph));
}

/* d(dU/dx)/da (tangent-linear only). */
static double potential_dx_da(const or_params *p, double x)
{
    const double ph = phase(p, x);
    const double k = 2.0 * M_PI / p->L;
    return -p->h * 0.453 * k * 2.0 * cos(2.0 * ph);
}

/* One explicit Euler-Maruyama step of Eqs. (ereservoir), (velocity) and
 * dx/dt = v; every right-hand side uses the values at step n.  s = (x, v, e). */
void or_em_step(const or_params *p, double dt, double z, double s[3])
{
    const double x = s[0], v = s[1], e = s[2];
    const double e_rate = p->q - p->c * e - p->d * e * v * v;
    const double v_rate = p->F0 + p->d * e * v - p->gamma0 * v - or_potential_dx(p, x);
    s[0] = x + dt * v;
    s[1] = v + dt * v_rate + sqrt(2.0 * p->D * dt) * z;
    s[2] = e + dt * e_rate;
}

/* Right-hand side of the drift of Eqs. (ereservoir), (velocity) and dx/dt = v at
 * s = (x, v, e): rate = (dx/dt, dv/dt, de/dt) without the noise. */
static void drift(const or_params *p, const double s[3], double rate[3])
{
    const double x = s[0], v = s[1], e = s[2];
    rate[0] = v;
    rate[1] = p->F0 + p->d * e * v - p->gamma0 * v - or_potential_dx(p, x);
    rate[2] = p->q - p->c * e - p->d * e * v * v;
}

/* One stochastic Heun step (the predictor-corrector, or improved Euler, scheme
 * for an SDE with additive noise; Kloeden & Platen, Numerical Solution of
 * Stochastic Differential Equations, 1992, Sec. 15.1): with the drift a(s) and
 * the velocity's noise increment w = sqrt(2 D dt) z of step n (one Gaussian
 * number, the same one the Euler-Maruyama step uses),
 *   predictor  s~ = s + a(s) dt + (0, w, 0)
 *   corrector  s' = s + (a(s) + a(s~)) dt / 2 + (0, w, 0).
 * Not the paper's scheme (Fig. 1 names none); offered beside it as a
 * higher-order variant.  *v_pred (may be NULL) receives the predictor's
 * velocity, so that x advances by (v + v~) dt / 2. */
void or_heun_step(const or_params *p, double dt, double z, double s[3], double *v_pred)
{
    const double w = sqrt(2.0 * p->D * dt) * z;
    double a0[3], a1[3], sp[3];
    drift(p, s, a0);
    sp[0] = s[0] + dt * a0[0];
    sp[1] = s[1] + dt * a0[1] + w;
    sp[2] = s[2] + dt * a0[2];
    drift(p, sp, a1);
    s[0] = s[0] + 0.5 * dt * (a0[0] + a1[0]);
    s[1] = s[1] + 0.5 * dt * (a0[1] + a1[1]) + w;
    s[2] = s[2] + 0.5 * dt * (a0[2] + a1[2]);
    if (v_pred)
        *v_pred = sp[1];
}

/* Tangent-linear of or_em_step along parameter direction dth =
 * (dD, dq, dc, dd, dgamma0, dasym), acting on the tangent state t = (dx, dv, de)
 * at the (pre-step) primal state s. */
static void tangent_step(const or_params *p, double dt, double z, const double s[3],
                         const double dth[6], double t[3])
{
    const double x = s[0], v = s[1], e = s[2];
    const double dx = t[0], dv = t[1], de = t[2];
    const double dD = dth[0], dq = dth[1], dc = dth[2], dd = dth[3], dg = dth[4], da = dth[5];
    const double sigma = sqrt(2.0 * p->D * dt);
    /* sigma grows like sqrt(D): at D = 0 its derivative in D does not exist, and
     * the D-direction of the tangent is undefined (NaN) from the first noise term on. */
    const double dsigma = (p->D > 0.0) ? dD * sigma / (2.0 * p->D) : (dD != 0.0 ? NAN : 0.0);
    const double de_rate = dq - dc * e - p->c * de - dd * e * v * v - p->d * de * v * v
                           - 2.0 * p->d * e * v * dv;
    const double dv_rate = dd * e * v + p->d * de * v + p->d * e * dv - dg * v - p->gamma0 * dv
                           - potential_dxx(p, x) * dx - potential_dx_da(p, x) * da;
    t[0] = dx + dt * dv;
    t[1] = dv + dt * dv_rate + dsigma * z;
    t[2] = de + dt * de_rate;
}

/* ------------------------------------------------------------------------ */
/* Marsaglia's xorshift generator with four 32-bit words of state (G. Marsaglia,
 * "Xorshift RNGs", J. Stat. Softw. 8(14), 2003; the variant with shifts
 * 11, 8, 19), the RNG of the paper's Fig. 1, kept as an option beside the
 * counter-based Philox stream.  One call advances the state (x, y, z, w) to
 * (y, z, w, w ^ (w >> 19) ^ t ^ (t >> 8)) with t = x ^ (x << 11) and returns
 * the new w.  Each trajectory seeds its own state from the Philox block of
 * counter 2^63 + 1 (the initial condition uses 2^63); an all-zero state (never
 * met in practice) becomes (0, 0, 0, 1).  Each step draws two words (u1, u2) and
 * uses the cosine branch of Box-Muller, one "xorshift, Box-Muller" per iteration
 * as in Fig. 1. */
uint32_t or_xorshift128_step(uint32_t s[4])
{
    const uint32_t t = s[0] ^ (s[0] << 11);
    s[0] = s[1];
    s[1] = s[2];
    s[2] = s[3];
    s[3] = s[3] ^ (s[3] >> 19) ^ t ^ (t >> 8);
    return s[3];
}

void or_xorshift_seed(uint64_t seed, uint64_t traj, uint32_t s[4])
{
    or_noise_words(seed, traj, ((uint64_t)1 << 63) + 1, s);
    if ((s[0] | s[1] | s[2] | s[3]) == 0)
        s[3] = 1;
}

/* The normal of the next step of an xorshift stream. */
double or_xorshift_normal(uint32_t s[4])
{
    double z[2];
    const uint32_t wa = or_xorshift128_step(s);
    const uint32_t wb = or_xorshift128_step(s);
    or_box_muller(wa, wb, z);
    return z[0];
}

/* Initial condition of global trajectory `traj` (counter m = 2^63). */
void or_initial_state(const or_params *p, uint64_t seed, int32_t v0_mode, uint64_t traj,
                      double s[3])
{
    uint32_t w[4];
    double z[2];
    or_noise_words(seed, traj, (uint64_t)1 << 63, w);
    s[0] = p->L * (double)(w[0] >> 8) * 0x1p-24;
    s[1] = 0.0;
    if (v0_mode == 1) {
        or_box_muller(w[1], w[2], z);
        s[1] = sqrt(p->D) * z[0];
    }
    s[2] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Ensemble run of one parameter set. */

typedef struct {
    or_params p;
    uint64_t seed;
    double dt;
    int64_t traj_base;      /* global id of the set's first trajectory */
    int64_t n_traj;
    int64_t n_steps;
    int64_t snapshot_every; /* 0: one snapshot after the last step */
    int32_t v0_mode;        /* 0: v0 = 0, 1: v0 ~ N(0, sqrt(D)) */
    int32_t n_threads;
    int32_t hist_x_bins;    /* 0: no position histogram */
    int32_t hist_v_bins;    /* 0: no velocity histogram */
    double v_lo, v_hi;
    int32_t want_grad;      /* Euler-Maruyama with Philox noise only */
    int32_t scheme;         /* 0: Euler-Maruyama (the paper's), 1: stochastic Heun */
    int32_t noise;          /* 0: Philox4x32-10 by (seed, trajectory, step); 1: xorshift per trajectory */
    int32_t reserved;
    int64_t grad_window;    /* W > 0: windowed gradient -- the tangents restart from zero at steps
                               W, 2W, ... (each window's time average differentiated with the state
                               at the window's start held fixed); 0: the full pathwise gradient */
} or_run_args;

typedef struct {
    double *x0, *x, *v, *e; /* [n_traj] final state, optional */
    double *vbar;           /* [n_traj] time-averaged velocity, optional */
    double *dvbar;          /* [n_traj][6] tangent of vbar, optional */
    uint64_t *hist_x;       /* [n_snap][hist_x_bins], optional */
    uint64_t *hist_v;       /* [n_snap][hist_v_bins + 2] (underflow, overflow last), optional */
    double sums[4];         /* sum vbar, sum vbar^2, sum dx, sum dx^2 */
    double grad[6];         /* d mean(vbar) / d(D, q, c, d, gamma0, asym) */
} or_run_out;

int64_t or_n_snapshots(int64_t n_steps, int64_t snapshot_every)
{
    if (snapshot_every <= 0)
        return 1;
    return n_steps / snapshot_every;
}

typedef struct {
    const or_run_args *a;
    int64_t lo, hi;
    double *x0, *x, *v, *e, *vbar, *dx, *dvbar;
    uint64_t *hx, *hv; /* private histograms */
} worker;

static void snapshot(const or_run_args *a, int64_t snap, const double s[3], uint64_t *hx,
                     uint64_t *hv)
{
    if (hx && a->hist_x_bins > 0) {
        const double L = a->p.L;
        const double xm = s[0] - L * floor(s[0] / L);
        int64_t b = (int64_t)floor(xm / L * (double)a->hist_x_bins);
        if (b < 0)
            b = 0;
        if (b >= a->hist_x_bins)
            b = a->hist_x_bins - 1;
        hx[snap * a->hist_x_bins + b] += 1;
    }
    if (hv && a->hist_v_bins > 0) {
        const int64_t B = a->hist_v_bins;
        int64_t b;
        if (s[1] < a->v_lo)
            b = B;
        else if (s[1] >= a->v_hi)
            b = B + 1;
        else {
            b = (int64_t)floor((s[1] - a->v_lo) / (a->v_hi - a->v_lo) * (double)B);
            if (b >= B)
                b = B - 1;
        }
        hv[snap * (B + 2) + b] += 1;
    }
}

static void *run_range(void *arg)
{
    worker *wk = (worker *)arg;
    const or_run_args *a = wk->a;
    const or_params *p = &a->p;
    static const double unit[6][6] = {{1, 0, 0, 0, 0, 0}, {0, 1, 0, 0, 0, 0}, {0, 0, 1, 0, 0, 0},
                                      {0, 0, 0, 1, 0, 0}, {0, 0, 0, 0, 1, 0}, {0, 0, 0, 0, 0, 1}};
    for (int64_t i = wk->lo; i < wk->hi; ++i) {
        const uint64_t traj = (uint64_t)(a->traj_base + i);
        double s[3];
        or_initial_state(p, a->seed, a->v0_mode, traj, s);
        const double x0 = s[0];
        double t[6][3];
        double tsum[6] = {0, 0, 0, 0, 0, 0};
        if (a->want_grad) {
            /* v0 = sqrt(D) z depends on D in mode 1. */
            for (int j = 0; j < 6; ++j)
                t[j][0] = t[j][1] = t[j][2] = 0.0;
            if (a->v0_mode == 1)
                t[0][1] = p->D > 0.0 ? s[1] / (2.0 * p->D) : NAN;
        }
        double vsum = 0.0;
        int64_t snap = 0;
        uint32_t xs[4];
        if (a->noise == 1)
            or_xorshift_seed(a->seed, traj, xs);
        if (a->n_steps == 0 && a->snapshot_every <= 0)
            snapshot(a, snap++, s, wk->hx, wk->hv);
        for (int64_t n = 0; n < a->n_steps; ++n) {
            const double z = a->noise == 1 ? or_xorshift_normal(xs) : or_normal(a->seed, traj, (uint64_t)n);
            if (a->scheme == 1) {
                /* x advances by (v + v~) dt / 2: that is the step's velocity */
                const double v_n = s[1];
                double v_pred;
                or_heun_step(p, a->dt, z, s, &v_pred);
                vsum += 0.5 * (v_n + v_pred);
            } else {
                vsum += s[1];
                if (a->want_grad) {
                    if (a->grad_window > 0 && n > 0 && n % a->grad_window == 0)
                        for (int j = 0; j < 6; ++j)
                            t[j][0] = t[j][1] = t[j][2] = 0.0;
                    for (int j = 0; j < 6; ++j) {
                        tsum[j] += t[j][1];
                        tangent_step(p, a->dt, z, s, unit[j], t[j]);
                    }
                }
                or_em_step(p, a->dt, z, s);
            }
            const int64_t done = n + 1;
            if (a->snapshot_every > 0 ? (done % a->snapshot_every == 0) : (done == a->n_steps))
                snapshot(a, snap++, s, wk->hx, wk->hv);
        }
        const double N = (double)a->n_steps;
        if (wk->x0)
            wk->x0[i] = x0;
        if (wk->x)
            wk->x[i] = s[0];
        if (wk->v)
            wk->v[i] = s[1];
        if (wk->e)
            wk->e[i] = s[2];
        wk->vbar[i] = a->n_steps > 0 ? vsum / N : 0.0;
        wk->dx[i] = s[0] - x0;
        if (a->want_grad)
            for (int j = 0; j < 6; ++j)
                wk->dvbar[i * 6 + j] = a->n_steps > 0 ? tsum[j] / N : 0.0;
    }
    return NULL;
}

/* Returns 0 on success, -1 on bad arguments, -2 on allocation failure. */
int or_run_set(const or_run_args *a, or_run_out *o)
{
    if (!a || !o || a->n_traj < 0 || a->n_steps < 0 || !(a->dt > 0.0) || !(a->p.L > 0.0)
        || a->p.D < 0.0 || a->hist_x_bins < 0 || a->hist_v_bins < 0
        || (a->hist_v_bins > 0 && !(a->v_hi > a->v_lo)) || a->scheme < 0 || a->scheme > 1
        || (a->scheme == 1 && a->want_grad) || a->noise < 0 || a->noise > 1 || (a->noise == 1 && a->want_grad)
        || a->grad_window < 0)
        return -1;
    const int64_t M = a->n_traj;
    const int64_t n_snap = or_n_snapshots(a->n_steps, a->snapshot_every);
    int nt = a->n_threads > 0 ? a->n_threads : 1;
    if (nt > 256)
        nt = 256;
    if ((int64_t)nt > M)
        nt = M > 0 ? (int)M : 1;

    double *vbar = o->vbar ? o->vbar : (double *)malloc(sizeof(double) * (size_t)(M + 1));
    double *dx = (double *)malloc(sizeof(double) * (size_t)(M + 1));
    double *dvbar = NULL;
    if (a->want_grad)
        dvbar = o->dvbar ? o->dvbar : (double *)malloc(sizeof(double) * 6 * (size_t)(M + 1));
    const size_t hx_len = (size_t)n_snap * (size_t)a->hist_x_bins;
    const size_t hv_len = (size_t)n_snap * (size_t)(a->hist_v_bins > 0 ? a->hist_v_bins + 2 : 0);
    uint64_t *hx_all = (o->hist_x && hx_len) ? (uint64_t *)calloc((size_t)nt * hx_len, 8) : NULL;
    uint64_t *hv_all = (o->hist_v && hv_len) ? (uint64_t *)calloc((size_t)nt * hv_len, 8) : NULL;
    worker *wk = (worker *)calloc((size_t)nt, sizeof(worker));
    pthread_t *th = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
    if (!vbar || !dx || (a->want_grad && !dvbar) || (o->hist_x && hx_len && !hx_all)
        || (o->hist_v && hv_len && !hv_all) || !wk || !th)
        return -2;

    for (int k = 0; k < nt; ++k) {
        wk[k].a = a;
        wk[k].lo = M * k / nt;
        wk[k].hi = M * (k + 1) / nt;
        wk[k].x0 = o->x0;
        wk[k].x = o->x;
        wk[k].v = o->v;
        wk[k].e = o->e;
        wk[k].vbar = vbar;
        wk[k].dx = dx;
        wk[k].dvbar = dvbar;
        wk[k].hx = hx_all ? hx_all + (size_t)k * hx_len : NULL;
        wk[k].hv = hv_all ? hv_all + (size_t)k * hv_len : NULL;
    }
    if (nt == 1) {
        run_range(&wk[0]);
    } else {
        for (int k = 0; k < nt; ++k)
            pthread_create(&th[k], NULL, run_range, &wk[k]);
        for (int k = 0; k < nt; ++k)
            pthread_join(th[k], NULL);
    }

    /* Ensemble sums in trajectory order (plain definition). */
    double s1 = 0, s2 = 0, s3 = 0, s4 = 0;
    for (int64_t i = 0; i < M; ++i) {
        s1 += vbar[i];
        s2 += vbar[i] * vbar[i];
        s3 += dx[i];
        s4 += dx[i] * dx[i];
    }
    o->sums[0] = s1;
    o->sums[1] = s2;
    o->sums[2] = s3;
    o->sums[3] = s4;
    for (int j = 0; j < 6; ++j) {
        double g = 0.0;
        if (a->want_grad)
            for (int64_t i = 0; i < M; ++i)
                g += dvbar[i * 6 + j];
        o->grad[j] = (a->want_grad && M > 0) ? g / (double)M : 0.0;
    }
    if (o->hist_x && hx_len) {
        memset(o->hist_x, 0, hx_len * 8);
        for (int k = 0; k < nt; ++k)
            for (size_t b = 0; b < hx_len; ++b)
                o->hist_x[b] += hx_all[(size_t)k * hx_len + b];
    }
    if (o->hist_v && hv_len) {
        memset(o->hist_v, 0, hv_len * 8);
        for (int k = 0; k < nt; ++k)
            for (size_t b = 0; b < hv_len; ++b)
                o->hist_v[b] += hv_all[(size_t)k * hv_len + b];
    }

    if (!o->vbar)
        free(vbar);
    free(dx);
    if (a->want_grad && !o->dvbar)
        free(dvbar);
    free(hx_all);
    free(hv_all);
    free(wk);
    free(th);
    return 0;
}
