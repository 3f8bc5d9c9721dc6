// abp_ctx.cuh -- definition of the opaque abp_ctx of the C ABI, shared by the
// runtime translation units (abp_api.cu, abp_adjoint.cu).  Not public.
#pragma once

#include <set>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "abp.h"
#include "abp_internal.cuh"

namespace abp {

constexpr int64_t kMaxSteps = (int64_t)1 << 34;  // counter blocks n >> 2 stay below 2^32

// A device allocation with a capacity (cap) and the size in use (bytes).
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    size_t bytes = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        bytes = 0;
    }
};

}  // namespace abp

struct abp_ctx {
    using DevBuf = abp::DevBuf;
    using Batch = abp::Batch;
    using State = abp::State;
    using Hist = abp::Hist;
    using Ckpt = abp::Ckpt;
    using Noise = abp::Noise;

    abp_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 0;
    std::string err;

    // batch (host mirror)
    bool have_batch = false;
    int32_t n_sets = 0;
    int32_t n_tiles = 0;
    int64_t total_traj = 0;
    int64_t max_steps = 0;
    int64_t g = 0;  // global steps issued: set s has done min(g, n_steps[s])
    bool ckpt_complete = true;  // adjoint checkpoints cover the run from step 0 (false after abp_load)
    bool adj_valid = false;     // the adjoint scratch holds the sums of the current run (abp_backward_traj)
    int ppt = 1;
    int sched = 1;                 // 1: lockstep launches, 2: work queue (autotuned when cfg.schedule = 0)
    int64_t steps_per_launch = 0;  // lockstep: steps per launch; work queue: steps per round
    std::string tune_report;       // the autotuner's candidates and choice for the batch (JSON text)
    int grid = 0;                  // work queue: resident blocks of the persistent launch
    int32_t hold_tile = -1;        // test hook (abp_test_hold_tile)
    int64_t wait_limit_ns = 60000000000LL;
    std::vector<int32_t> perm;     // tiles by decreasing step count
    std::vector<int64_t> perm_steps;
    // CUDA graphs of repeated work-queue windows
    struct GraphEntry {
        int sched;
        int64_t kernels;  // kernels per replay
        int64_t g0, g1, seg;
        uint64_t seed, traj_base;
        int32_t hold;
        int64_t wait_limit_ns;
        int32_t n_items;
        void *round_start;  // device copy owned by the entry
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    std::set<std::pair<int64_t, int64_t>> windows_seen;  // windows run once, not yet captured
    int64_t n_snap = 0;
    int64_t n_ckpt = 0;
    int64_t launches = 0;  // kernels enqueued by this context
    std::vector<abp_params> params;
    std::vector<int64_t> n_traj, n_steps;
    std::vector<int32_t> set_tile_begin, tile_count, tile_set, set_packed, set_order, slot_set;
    std::vector<int64_t> tile_first, set_first;
    int32_t n_single = 0;  // tiles [n_single, n_tiles) are packed
    int32_t n_unpacked = 0;  // sets in one-set tiles
    int32_t narrow = 0, sub_single = 1, sub_packed = 1;  // narrow lockstep launch (small batches)

    // device
    DevBuf d_params, d_steps, d_set_tile_begin, d_tile_first, d_tile_count, d_tile_set, d_set_first, d_set_order,
        d_slot_set;
    DevBuf d_coef;  // per-set step coefficients (coef_tables)
    // Page-locked host staging of the batch tables abp_set_params uploads (one
    // allocation, grown when a batch needs more; copies from pageable memory cost
    // a fixed fraction of a millisecond each on this platform).
    void *h_stage = nullptr;
    size_t h_stage_cap = 0;
    DevBuf d_y, d_yacc, d_ylo, d_v, d_e, d_y0, d_cell, d_xs;
    DevBuf d_hx, d_hv, d_ckpt, d_partials, d_moments, d_status;
    DevBuf d_queue, d_round, d_perm;  // work queue: head + done[n_tiles]; round starts; tile order
    DevBuf d_adj;  // adjoint scratch
    cudaStream_t aux = nullptr;  // second stream of abp_backward (level-1 re-runs beside the reverse sweep)
    cudaEvent_t adj_ev[5] = {};  // its ordering events

    // Live results (abp_live): snapshot k is copied to the caller's page-locked
    // buffers on live_stream once the main stream has passed step (k + 1) S.
    static constexpr int kLiveRing = 64;  // events kept for snapshots in flight
    bool live = false;
    double *live_mom = nullptr;
    uint32_t *live_hx = nullptr, *live_hv = nullptr;
    int64_t live_sent = 0, live_ready = 0;  // snapshots enqueued / known to have arrived
    cudaStream_t live_stream = nullptr;
    cudaEvent_t live_done[kLiveRing] = {}, live_copied[kLiveRing] = {};
    DevBuf d_live_mom;  // [n_snap][n_sets][8] moments at the snapshot steps

    Batch batch() const {
        Batch b;
        b.n_sets = n_sets;
        b.n_tiles = n_tiles;
        b.n_single = n_single;
        b.total_traj = total_traj;
        b.set_first = n_single < n_tiles ? (const int64_t *)d_set_first.p : nullptr;
        b.set_order = n_unpacked < n_sets ? (const int32_t *)d_set_order.p : nullptr;
        b.slot_set = n_single < n_tiles ? (const int32_t *)d_slot_set.p : nullptr;
        b.n_unpacked = n_unpacked;
        b.narrow = narrow;
        b.sub_single = sub_single;
        b.sub_packed = sub_packed;
        b.params = (const abp_params *)d_params.p;
        b.set_steps = (const int64_t *)d_steps.p;
        b.set_tile_begin = (const int32_t *)d_set_tile_begin.p;
        b.tile_first = (const int64_t *)d_tile_first.p;
        b.tile_count = (const int32_t *)d_tile_count.p;
        b.tile_set = (const int32_t *)d_tile_set.p;
        b.dbg = (int32_t *)d_status.p;
        if (d_coef.bytes) abp::coef_tables(d_coef.p, n_sets, &b.coef_f, &b.coef_d);
        return b;
    }
    State state() const {
        State s;
        s.fp64 = cfg.state_fp64 != 0;
        s.y = d_y.p;
        s.yacc = d_yacc.p;
        s.ylo = d_ylo.p;
        s.v = d_v.p;
        s.e = d_e.p;
        s.y0 = d_y0.p;
        s.cell = (int32_t *)d_cell.p;
        s.xs = cfg.noise == 1 ? (uint4 *)d_xs.p : nullptr;
        return s;
    }
    Hist hist() const {
        Hist h;
        h.x = (uint32_t *)d_hx.p;
        h.v = (uint32_t *)d_hv.p;
        h.bx = cfg.hist_x_bins;
        h.bv = cfg.hist_v_bins;
        h.v_lo = cfg.v_lo;
        h.v_hi = cfg.v_hi;
        h.snap_every = cfg.snapshot_every;
        h.n_snap = n_snap;
        return h;
    }
    Ckpt ckpt() const {
        Ckpt c;
        c.ck = (float4 *)d_ckpt.p;
        c.every = cfg.checkpoint_every;
        c.n_slots = n_ckpt;
        return c;
    }
    Noise noise() const {
        Noise n;
        n.k0 = (uint32_t)cfg.seed;
        n.k1 = (uint32_t)(cfg.seed >> 32);
        n.dt = cfg.dt;
        n.v0_mode = cfg.v0_mode;
        n.traj_base = cfg.traj_base;
        n.scheme = cfg.scheme;
        n.noise = cfg.noise;
        return n;
    }
    void drop_graphs() {
        for (GraphEntry &g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.round_start) cudaFree(g.round_start);
        }
        graphs.clear();
        windows_seen.clear();
    }
    void release_batch() {
        // Buffers are kept (and reused by the next batch when large enough);
        // see release_all() for freeing them.  Live results stop: their
        // buffers were sized by the batch.
        if (live_stream) cudaStreamSynchronize(live_stream);
        drop_graphs();
        have_batch = false;
        adj_valid = false;
        live = false;
        live_mom = nullptr;
        live_hx = live_hv = nullptr;
        live_sent = live_ready = 0;
    }
    void release_streams() {
        if (live_stream) cudaStreamSynchronize(live_stream);
        for (cudaEvent_t *arr : {adj_ev + 0, live_done + 0, live_copied + 0}) {
            const int n = arr == adj_ev ? 5 : kLiveRing;
            for (int i = 0; i < n; ++i)
                if (arr[i]) {
                    cudaEventDestroy(arr[i]);
                    arr[i] = nullptr;
                }
        }
        if (live_stream) {
            cudaStreamDestroy(live_stream);
            live_stream = nullptr;
        }
        if (aux) {
            cudaStreamDestroy(aux);
            aux = nullptr;
        }
    }
    void release_all() {
        if (live_stream) cudaStreamSynchronize(live_stream);
        drop_graphs();
        for (DevBuf *b : {&d_queue, &d_round, &d_perm, &d_set_first, &d_set_order, &d_slot_set, &d_params, &d_coef, &d_steps, &d_set_tile_begin, &d_tile_first, &d_tile_count, &d_tile_set, &d_y,
                          &d_yacc, &d_ylo, &d_v, &d_e, &d_y0, &d_cell, &d_xs, &d_hx, &d_hv, &d_ckpt, &d_partials,
                          &d_moments, &d_adj, &d_live_mom})
            b->release();
        if (h_stage) cudaFreeHost(h_stage);
        h_stage = nullptr;
        h_stage_cap = 0;
        have_batch = false;
        live = false;
    }
};

