// abp_internal.cuh -- device-side views shared by the C-ABI runtime
// (abp_api.cu) and the kernels (abp_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "abp.h"

namespace abp {

// Trajectories per CUDA block of the integrator and the per-tile kernels.
constexpr int kThreads = 256;
// Steps between position folds (yacc into y, whole periods into cell).  Folds
// happen at absolute step multiples, so any split of a run into launches gives
// bitwise identical arithmetic.
constexpr int kBlockSteps = 64;

// One batch of parameter sets, tiled for the device.  Tiles [0, n_single) are
// contiguous runs of at most kThreads * ppt trajectories of one set (the tiles
// of a set are consecutive).  Tiles [n_single, n_tiles) are packed: each holds
// at most kThreads trajectories of several small sets with equal step counts
// (whole sets, consecutive in set order), one trajectory per thread.
struct Batch {
    int32_t n_sets;
    int32_t n_tiles;
    int32_t n_single;
    int64_t total_traj;
    const int64_t *set_first;      // [n_sets + 1] first trajectory of each set (packed batches; else NULL)
    const int32_t *set_order;      // [n_sets] sets in one-set tiles, then sets in packed tiles (NULL: all one-set, in order)
    const int32_t *slot_set;       // [n_tiles - n_single][kThreads] set of each packed-tile slot (NULL: no packed tiles)
    int32_t n_unpacked;            // sets in one-set tiles (the first n_unpacked entries of set_order)
    // Narrow launch of the lockstep integrator (small batches): blocks of `narrow`
    // threads (0: off), one trajectory per thread, sub_single blocks per one-set
    // tile and sub_packed per packed tile.  Tiles, and so every result, are the same.
    int32_t narrow, sub_single, sub_packed;
    const abp_params *params;      // [n_sets]
    const int64_t *set_steps;      // [n_sets] steps to run
    const int32_t *set_tile_begin; // [n_sets + 1]
    const int64_t *tile_first;     // [n_tiles] first global trajectory id (= state index)
    const int32_t *tile_count;     // [n_tiles] trajectories in the tile (>= 1)
    const int32_t *tile_set;       // [n_tiles] the set (packed tile: its first set)
    int32_t *dbg = nullptr;        // status word of the checked build (ABP_DEBUG_CHECKS)
    // Per-set step coefficients, Coef<float> / Coef<double> [n_sets], formed once per batch
    // (coef_kernel); NULL: each kernel forms them from params itself (same function).
    const void *coef_f = nullptr, *coef_d = nullptr;
};

// Checked build (-DABP_DEBUG_CHECKS=1, the stand-in for a memory checker): an
// index outside [0, n) records status 3 in *st and is replaced by 0, so the
// access stays inside its buffer and the launch runs to its end; the host
// then reports ABP_ESTATE.  Release builds compile the check away.
#ifndef ABP_DEBUG_CHECKS
#define ABP_DEBUG_CHECKS 0
#endif
__device__ __forceinline__ int64_t dchk(int64_t i, int64_t n, int32_t *st) {
#if ABP_DEBUG_CHECKS
    if (i < 0 || i >= n) {
        if (st) atomicCAS(st, 0, 3);
        return 0;
    }
#endif
    (void)n;
    (void)st;
    return i;
}

// Structure-of-arrays trajectory state.  Element type is float (fp64 = false)
// or double (fp64 = true) for y, yacc, ylo, v, e, y0.
// x = L (cell + y + yacc + ylo); the time-averaged velocity of n steps is
// (x_n - x_0) / (n dt), since the scheme advances x by v_k dt at every step.
struct State {
    bool fp64;
    void *y;       // fraction of the period
    void *yacc;    // increments v dt / L of the open block of kBlockSteps steps
    void *ylo;     // rounding errors of the folds (displacement only)
    void *v;       // velocity
    void *e;       // depot energy
    void *y0;      // initial fraction (x0 = L y0)
    int32_t *cell; // period index
    uint4 *xs;     // xorshift state (x, y, z, w) of each trajectory (noise 1), else NULL
};

struct Hist {
    uint32_t *x;         // [n_snap][n_sets][bx]
    uint32_t *v;         // [n_snap][n_sets][bv + 2]
    int32_t bx, bv;
    double v_lo, v_hi;
    int64_t snap_every;  // 0: after the last step of each set
    int64_t n_snap;
};

// Checkpoints for the adjoint: state after steps 0, K, 2K, ... as
// (y, yacc, v, e) -- everything the dynamics read -- slot-major:
// ck[slot * total_traj + traj].
struct Ckpt {
    float4 *ck;
    int64_t every;  // 0: none
    int64_t n_slots;
};

struct Noise {
    uint32_t k0, k1;     // Philox key = seed
    double dt;
    int32_t v0_mode;
    uint64_t traj_base;  // added to every state index to give the global trajectory id
    uint32_t rk[20];     // round keys: rk[2r], rk[2r+1] = (k0 + r W0, k1 + r W1)
    int32_t scheme;      // 0 Euler-Maruyama, 1 stochastic Heun (FP32 state)
    int32_t noise;       // 0 Philox by (seed, trajectory, step), 1 xorshift per trajectory
};

// Work queue of the persistent integrator (device buffers owned by the context).
struct Queue {
    int32_t *head;              // next item to pop
    int32_t *done;              // [n_tiles] rounds of the window each tile has published
    int32_t *status;            // 0 ok; 1 a dependency wait exceeded wait_limit_ns
    const int32_t *round_start; // [n_rounds + 1] first item of each round
    const int32_t *perm;        // [n_tiles] tiles by decreasing step count (stable)
    int32_t n_rounds;
    int32_t n_items;
    int32_t hold_tile;          // test hook: this tile never publishes its rounds (-1: none)
    int64_t wait_limit_ns;
};

// Derived moments of one set (Sec. 2: averages over noise realisations) from its four
// FP64 sums a = (sum vbar, sum vbar^2, sum dx, sum dx^2) over M trajectories of n steps
// of length dt, into o[8] in the layout of abp_reduce.  Host and device run the same
// correctly rounded operations in the same order (no fused multiply-add on either side),
// so a set gives the same bits whether its moments are formed by a reduction kernel, by
// the combining kernel or on the host.
__host__ __device__ inline double mom_mul(double x, double y) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(x, y);
#else
    return x * y;
#endif
}
__host__ __device__ inline double mom_sub(double x, double y) {
#ifdef __CUDA_ARCH__
    return __dsub_rn(x, y);
#else
    return x - y;
#endif
}
__host__ __device__ inline void moments_from_sums(double *o, const double *a, int64_t M, int64_t n, double dt) {
    const double Md = (double)M;
    const double mean_v = M > 0 ? a[0] / Md : 0.0;
    const double var_v = M > 1 ? mom_sub(a[1], mom_mul(mom_mul(Md, mean_v), mean_v)) / (Md - 1.0) : 0.0;
    const double msd = M > 0 ? a[3] / Md : 0.0;
    const double mdx = M > 0 ? a[2] / Md : 0.0;
    const double T = mom_mul((double)n, dt);
    o[0] = mean_v;
    o[1] = M > 0 ? sqrt((var_v > 0.0 ? var_v : 0.0) / Md) : 0.0;
    o[2] = msd;
    o[3] = T > 0.0 ? mom_sub(msd, mom_mul(mdx, mdx)) / mom_mul(2.0, T) : 0.0;
    for (int j = 0; j < 4; ++j) o[4 + j] = a[j];
}

// Where a caller's pointer points, seen from device `dev`: host memory (pageable
// or page-locked; the library copies to and from it), memory that kernels on `dev`
// may read and write (that device's own memory, or managed memory), or another
// GPU's memory, which the entry points reject: a kernel storing to it would write
// to a peer device or fault.
enum class PtrKind { Host, Device, OtherDevice };
inline PtrKind ptr_kind(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return PtrKind::Host;
    }
    if (a.type == cudaMemoryTypeManaged) return PtrKind::Device;
    if (a.type != cudaMemoryTypeDevice) return PtrKind::Host;
    return a.device == dev ? PtrKind::Device : PtrKind::OtherDevice;
}
// The device address of page-locked host memory that kernels may write (mapped into
// the device's address space), else NULL.
template <typename T>
inline T *mapped_host(T *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? static_cast<T *>(a.devicePointer) : nullptr;
}
inline int current_device() {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return d;
}

// Columns 0..3 of moments [n][8] from its columns 4..7, set i having M[i]
// trajectories of N[i] steps (host arrays, copied into the launches).
cudaError_t launch_combine_moments(int32_t n, double *moments, const int64_t *M, const int64_t *N, double dt,
                                   cudaStream_t st);

cudaError_t launch_init(const Batch &b, const State &s, const Hist &h, const Ckpt &c, const Noise &nz,
                        cudaStream_t st);
// NVTX range over one C ABI call (nested ranges of the calling thread), for
// profilers that trace the host timeline; without a tool attached the push
// and pop return at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Device-side waits of a lockstep launch (the warp-specialised narrow form):
// the context's status word, the wait limit and the test hook's held tile.
struct WaitCtl {
    int32_t *status;
    int64_t limit_ns;
    int32_t hold_tile;  // test hook: this tile's producer warps never hand over noise (-1: none)
};

cudaError_t launch_integrate(const Batch &b, const State &s, const Hist &h, const Ckpt &c, const Noise &nz,
                             int ppt, int64_t g0, int64_t g1, cudaStream_t st, const WaitCtl *wait = nullptr);
// partials: [n_tiles][4] scratch; moments: [n_sets][8].
// The per-set coefficient tables of a batch in one device buffer of coef_table_bytes(n)
// bytes: coef_tables gives the two tables inside it, launch_coef fills them from the
// device parameter array (the step's FP64 set-up done once per batch instead of at the
// start of every window, work item and block).
size_t coef_table_bytes(int32_t n_sets);
void coef_tables(void *buf, int32_t n_sets, const void **coef_f, const void **coef_d);
cudaError_t launch_coef(const abp_params *params, int32_t n_sets, double dt, void *buf, cudaStream_t st);

cudaError_t launch_reduce(const Batch &b, const State &s, const Noise &nz, int64_t g, double *partials,
                          double *moments, cudaStream_t st);
cudaError_t launch_get_state(const Batch &b, const State &s, double dt, int64_t g, double *x, double *x0, double *v,
                             double *e, double *vbar, cudaStream_t st);
cudaError_t launch_philox(uint32_t k0, uint32_t k1, const uint64_t *traj, const uint64_t *m, int64_t n,
                          uint32_t *out, cudaStream_t st);
cudaError_t launch_xorshift(uint32_t k0, uint32_t k1, uint64_t traj, int64_t count, uint32_t *out, cudaStream_t st);
cudaError_t launch_normals(uint32_t k0, uint32_t k1, uint64_t traj, uint64_t n0, int64_t count, float *out,
                           cudaStream_t st);

cudaError_t launch_persistent(const Batch &b, const State &s, const Hist &h, const Ckpt &c, const Noise &nz,
                              const Queue &q, int ppt, int grid, int64_t g0, int64_t g1, int64_t seg,
                              cudaStream_t st);
// Resident blocks per SM of the persistent integrator (sets its shared-memory limit too).
// mode: 0 Euler-Maruyama, 1 stochastic Heun, 2 Euler-Maruyama with xorshift noise
cudaError_t persistent_occupancy(bool fp64, int ppt, size_t smem, int *blocks_per_sm, int mode = 0);
cudaError_t integrate_occupancy(bool fp64, int ppt, size_t smem, int *blocks_per_sm, int mode = 0);

}  // namespace abp
