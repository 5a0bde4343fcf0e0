// Internal state of the C ABI's forest object and the helpers shared by the
// translation units that launch kernels.  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/amr.h"
#include "common.cuh"
#include "forest.hpp"
#include "pattern.hpp"
#include "stage.cuh"

namespace amrb {

struct DBuf {
    void *p = nullptr;
    size_t cap = 0;
};

// one timed device phase: events recorded on the launch stream around it
struct TraceRec {
    int phase;
    cudaEvent_t a, b;
};

}  // namespace amrb

struct amr_forest {
    amr_config cfg{};                 // shared settings; max_blocks = total capacity
    std::vector<amr_config> icfg;     // per instance
    std::vector<amrb::Forest> inst;         // per instance; blocks numbered consecutively
    std::vector<int64_t> offset;      // first block of each instance, total at the end
    uint64_t revision = 1;            // bumped whenever any instance's mesh changes
    amrb::Pattern pat;
    uint64_t pattern_rev = ~0ull;
    amrb::Geom geom{};
    int esize = 8;
    size_t block_bytes = 0;
    void *state = nullptr;
    amrb::DBuf r1, r2, r1g, r3, info, fix, fix_start, bflux, bcdata, sc, partial, sums, flags, ops, level;
    amrb::DBuf dxtab, invdxtab, bctype, bcval, cfltab, ranges;   // per-instance tables
    amrb::DBuf feat, prob, mflags, flist;                        // learned-flag predictor
    amrb::DBuf slist;                                           // criterion: FP32 screen count + FP64 list
    amrb::DBuf wflux;                                            // WENO5 stage scratch (face fluxes)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    uint64_t graph_rev = ~0ull;
    int64_t graph_nodes = 0;
    int graph_flags = -1;
    bool scalar_stage = false;   // per-cell FP32 kernel instead of a pair kernel (tuning choice)
    int items_per_cta = 1;       // stage launch: CTAs loop over this many (block, tile) items
    bool persistent = false;     // stage launch: grid = SMs x resident CTAs, grid-stride sweep
    int pair_tile = 0;           // FP32 pair kernel staging tile: 0 default (16, N for N = 8), or 8
    int n_sms = 0;
    int64_t launches = 0;
    bool tracing = false;                      // per-phase timing on (steps then run without a graph)
    std::vector<cudaEvent_t> ev_free;          // timing events ready for reuse
    std::vector<amrb::TraceRec> trace_open;    // recorded phases not yet added to the totals
    bool trace_lost = false;                   // a phase went untimed since the last read with reset
    double trace_ms[AMR_N_PHASES] = {};
    int64_t trace_n[AMR_N_PHASES] = {};
    std::string err;
};

namespace amrb {

inline amr_status fail(amr_forest *f, amr_status s, const char *fmt, ...) {
    if (f) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        f->err = buf;
    }
    return s;
}

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(f, AMR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

inline int64_t nblocks(const amr_forest *f) { return f->offset.empty() ? 0 : f->offset.back(); }

// WENO5 stages of FP32 3D blocks of 8^3 or 16^3 cells run as one kernel
// (k_weno_fused), which can gather same-level halos; the others run the
// two passes on filled ghost cells
inline bool weno_fused_applies(const amr_forest *f) {
    return f->cfg.precision == 32 && f->cfg.ndim == 3 && (f->cfg.block_n == 8 || f->cfg.block_n == 16);
}
inline int n_inst(const amr_forest *f) { return int(f->inst.size()); }

// ---- per-phase timing (tracing): device phases by CUDA events, host phases
// by the wall clock
// adds every recorded phase to the totals; false if some record could not
// be timed (it is dropped)
inline bool trace_drain(amr_forest *f) {
    bool ok = true;
    for (const TraceRec &t : f->trace_open) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.b) == cudaSuccess && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            f->trace_ms[t.phase] += double(ms);
            f->trace_n[t.phase] += 1;
        } else {
            ok = false;
        }
        f->ev_free.push_back(t.a);
        f->ev_free.push_back(t.b);
    }
    f->trace_open.clear();
    return ok;
}

inline cudaEvent_t trace_event(amr_forest *f) {
    if (!f->ev_free.empty()) {
        cudaEvent_t e = f->ev_free.back();
        f->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}

// Times the launches issued during its lifetime on stream st as one record of
// `phase`; does nothing unless tracing is on and st is not being captured.
class TraceSpan {
  public:
    TraceSpan(amr_forest *f, int phase, cudaStream_t st) : f_(f), st_(st), phase_(phase) {
        if (!f->tracing) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            cudaGetLastError();
            f->trace_lost = true;
            return;
        }
        if (cs != cudaStreamCaptureStatusNone) return;   // a captured phase is timed by its replays, not here
        a_ = trace_event(f);
        if (a_ && cudaEventRecord(a_, st) != cudaSuccess) {
            cudaGetLastError();
            f->ev_free.push_back(a_);
            a_ = nullptr;
        }
        if (!a_) f->trace_lost = true;   // this phase goes untimed: amr_trace_read reports it
    }
    ~TraceSpan() {
        if (!a_) return;
        cudaEvent_t b = trace_event(f_);
        if (!b || cudaEventRecord(b, st_) != cudaSuccess) {
            cudaGetLastError();
            f_->ev_free.push_back(a_);
            if (b) f_->ev_free.push_back(b);
            f_->trace_lost = true;
            return;
        }
        f_->trace_open.push_back({phase_, a_, b});
        // bounded: a long traced run syncs now and then; a record that could
        // not be timed there is reported by the next amr_trace_read
        if (f_->trace_open.size() >= 4096 && !trace_drain(f_)) f_->trace_lost = true;
    }
    TraceSpan(const TraceSpan &) = delete;
    TraceSpan &operator=(const TraceSpan &) = delete;

  private:
    amr_forest *f_;
    cudaStream_t st_;
    int phase_;
    cudaEvent_t a_ = nullptr;
};

class HostSpan {
  public:
    HostSpan(amr_forest *f, int phase) : f_(f), phase_(phase), t0_(std::chrono::steady_clock::now()) {}
    ~HostSpan() {
        if (!f_->tracing) return;
        f_->trace_ms[phase_] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0_).count();
        f_->trace_n[phase_] += 1;
    }
    HostSpan(const HostSpan &) = delete;
    HostSpan &operator=(const HostSpan &) = delete;

  private:
    amr_forest *f_;
    int phase_;
    std::chrono::steady_clock::time_point t0_;
};

// grid of a stage launch for `items` (block, tile) items under the forest's tuning
inline int64_t stage_grid(const amr_forest *f, int64_t items, int occupancy) {
    if (f->persistent) return std::max<int64_t>(1, std::min<int64_t>(items, int64_t(f->n_sms) * std::max(occupancy, 1)));
    return (items + f->items_per_cta - 1) / f->items_per_cta;
}
inline void *slot_ptr(const amr_forest *f, int s) { return static_cast<char *>(f->state) + size_t(s) * f->cfg.max_blocks * f->block_bytes; }

// Kernel launchers, each instantiated in its own translation unit so that the
// library builds in parallel.
template <class real, int D>
amr_status launch_ghosts(amr_forest *f, int s, cudaStream_t st, bool gather);
template <class real, int D, int N, int NG, bool GEN, int PH>
amr_status launch_stage_t(amr_forest *f, const StageArgs<real> &a, cudaStream_t st);
template <int D, int N, int FLX>
amr_status launch_stage_pair(amr_forest *f, const StageArgs<float> &a, cudaStream_t st);
template <int D, int N>
amr_status launch_adv_pair(amr_forest *f, const StageArgs<float> &a, cudaStream_t st);
template <class real, int D, int PH>
amr_status launch_weno(amr_forest *f, const StageArgs<real> &a, real *flux, cudaStream_t st);

}  // namespace amrb
