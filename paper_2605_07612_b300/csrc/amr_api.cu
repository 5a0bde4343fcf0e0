// C ABI of the B300 block-AMR library (declared in include/amr.h).
// Host orchestration only: every arithmetic step of the hot path runs in the
// kernels of ghost.cuh, stage.cuh and misc.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <memory>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "api_internal.cuh"
#include "misc.cuh"
#include "mlp.cuh"

using namespace amrb;

namespace {

void *dev_alloc(amr_forest *f, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (f->cfg.dev_alloc) return f->cfg.dev_alloc(bytes, f->cfg.alloc_ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(amr_forest *f, void *p) {
    if (!p) return;
    if (f->cfg.dev_free) f->cfg.dev_free(p, f->cfg.alloc_ctx);
    else cudaFree(p);
}

amr_status ensure(amr_forest *f, DBuf &b, size_t bytes) {
    if (b.cap >= bytes && b.p) return AMR_OK;
    size_t want = std::max<size_t>(bytes + bytes / 4, 256);
    void *p = dev_alloc(f, want);
    if (!p) return fail(f, AMR_ENOMEM, "device allocation of %zu bytes failed", want);
    dev_free(f, b.p);
    b.p = p;
    b.cap = want;
    f->graph_rev = ~0ull;   // pointers moved: a captured graph is stale
    return AMR_OK;
}

template <class T>
amr_status upload(amr_forest *f, DBuf &b, const std::vector<T> &v) {
    amr_status s = ensure(f, b, sizeof(T) * std::max<size_t>(v.size(), 1));
    if (s != AMR_OK) return s;
    if (!v.empty()) CU(cudaMemcpy(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return AMR_OK;
}



void set_offsets(amr_forest *f) {
    f->offset.assign(1, 0);
    for (const Forest &F : f->inst) f->offset.push_back(f->offset.back() + int64_t(F.leaves.size()));
}

const Leaf &leaf_at(const amr_forest *f, int64_t b, int *which = nullptr) {
    size_t i = size_t(std::upper_bound(f->offset.begin(), f->offset.end(), b) - f->offset.begin()) - 1;
    if (which) *which = int(i);
    return f->inst[i].leaves[size_t(b - f->offset[i])];
}


void fill_geom(amr_forest *f) {
    const amr_config &c = f->cfg;
    Geom &g = f->geom;
    g.N = c.block_n;
    g.ng = c.n_ghost;
    g.S = c.block_n + 2 * c.n_ghost;
    g.D = c.ndim;
    g.V = c.n_var;
    g.ncell = 1;
    for (int d = 0; d < c.ndim; ++d) g.ncell *= g.S;
    g.bstride = g.ncell * g.V;
    g.phys = c.physics;
    for (int d = 0; d < 3; ++d) g.vel[d] = d < c.ndim ? c.velocity[d] : 0.0;
}

// cell sizes per (instance, level), boundary kinds/values and CFL numbers per
// instance, uploaded once at creation
amr_status upload_tables(amr_forest *f) {
    const int ni = n_inst(f);
    std::vector<double> dx(static_cast<size_t>(ni) * kMaxLevels * 3), idx(dx.size()), cfl(static_cast<size_t>(ni));
    std::vector<int32_t> bct(size_t(ni) * 6);
    std::vector<double> bcv(size_t(ni) * 48);
    for (int i = 0; i < ni; ++i) {
        const amr_config &c = f->icfg[size_t(i)];
        for (int l = 0; l < kMaxLevels; ++l)
            for (int d = 0; d < 3; ++d) {
                // same evaluation order as a plain len / ntrees / (N 2^l)
                const double h = c.len[d] / double(c.ntrees[d]) / (double(c.block_n) * double(1ll << l));
                dx[(size_t(i) * kMaxLevels + l) * 3 + d] = h;
                idx[(size_t(i) * kMaxLevels + l) * 3 + d] = 1.0 / h;
            }
        cfl[size_t(i)] = c.cfl;
        for (int q = 0; q < 6; ++q) {
            bct[size_t(i) * 6 + q] = c.bc[q];
            for (int v = 0; v < 8; ++v) bcv[(size_t(i) * 6 + q) * 8 + v] = c.bc_val[q][v];
        }
    }
    amr_status s;
    if ((s = upload(f, f->dxtab, dx)) != AMR_OK) return s;
    if ((s = upload(f, f->invdxtab, idx)) != AMR_OK) return s;
    if ((s = upload(f, f->cfltab, cfl)) != AMR_OK) return s;
    if ((s = upload(f, f->bctype, bct)) != AMR_OK) return s;
    if (f->cfg.precision == 64) {
        if ((s = upload(f, f->bcval, bcv)) != AMR_OK) return s;
    } else {
        std::vector<float> b32(bcv.begin(), bcv.end());
        if ((s = upload(f, f->bcval, b32)) != AMR_OK) return s;
    }
    f->geom.dx = static_cast<const double *>(f->dxtab.p);
    f->geom.inv_dx = static_cast<const double *>(f->invdxtab.p);
    return AMR_OK;
}

amr_status validate(const amr_config *c, std::string &why) {
    char b[256];
    auto bad = [&](const char *m) { why = m; return AMR_EINVAL; };
    if (c->ndim != 2 && c->ndim != 3) return bad("ndim must be 2 or 3");
    if (c->block_n != 8 && c->block_n != 16 && c->block_n != 32) return bad("block_n must be 8, 16 or 32");
    if (c->n_ghost < 1 || c->n_ghost > 4) return bad("n_ghost must be 1..4");
    if (c->block_n < 2 * c->n_ghost) return bad("block_n must be >= 2 n_ghost");
    if (c->physics != AMR_PHYS_EULER && c->physics != AMR_PHYS_ADVECTION) return bad("unknown physics");
    if (c->physics == AMR_PHYS_EULER && c->n_var != c->ndim + 2) return bad("n_var must be ndim + 2 (Euler)");
    if (c->physics == AMR_PHYS_ADVECTION) {
        if (c->n_var != 1) return bad("n_var must be 1 (scalar advection)");
        for (int d = 0; d < 3; ++d) {
            if (!std::isfinite(c->velocity[d])) return bad("velocity must be finite");
            if (c->gravity[d] != 0.0) return bad("scalar advection has no gravity source");
        }
    }
    if (c->max_level < 0 || c->max_level >= kMaxLevels) return bad("max_level must be 0..12");
    if (c->max_blocks < 1 || c->n_states < 1) return bad("max_blocks and n_states must be >= 1");
    if (c->precision != 32 && c->precision != 64) return bad("precision must be 32 or 64");
    if (c->limiter < AMR_LIM_MINMOD || c->limiter > AMR_LIM_UPWIND) return bad("unknown limiter");
    if (c->limiter == AMR_LIM_WENO5 && c->n_ghost < 3) return bad("WENO5 needs n_ghost >= 3");
    if (c->flux < AMR_FLUX_RUSANOV || c->flux > AMR_FLUX_HLL) return bad("unknown flux");
    if (!(c->gamma > 1.0) || !(c->cfl > 0.0)) return bad("gamma must be > 1 and cfl > 0");
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(c->gravity[d])) return bad("gravity must be finite");
    for (int d = 0; d < c->ndim; ++d) {
        if (c->ntrees[d] < 1 || (int64_t(c->ntrees[d]) << c->max_level) >= (1 << 19)) return bad("ntrees x 2^max_level must be < 2^19");
        if (!(c->len[d] > 0.0)) return bad("len must be > 0");
        for (int s = 0; s < 2; ++s) {
            int t = c->bc[2 * d + s];
            if (!c->periodic[d] && (t < 1 || t > 3)) {
                snprintf(b, sizeof b, "face %d of a non-periodic dimension needs a Dirichlet/Neumann/data boundary", 2 * d + s);
                why = b;
                return AMR_EINVAL;
            }
        }
    }
    return AMR_OK;
}

// ------------------------------------------------------------ pattern upload
amr_status upload_pattern(amr_forest *f) {
    if (f->pattern_rev == f->revision) return AMR_OK;
    HostSpan span(f, AMR_PHASE_PATTERN_HOST);
    std::string why;
    std::vector<const Forest *> ptrs;
    for (const Forest &F : f->inst) ptrs.push_back(&F);
    if (!build_pattern(ptrs, f->offset, f->pat, why, f->cfg.diagonal_ghosts != 0)) return fail(f, AMR_ESTATE, "%s", why.c_str());
    if (f->cfg.host_only) {
        f->pattern_rev = f->revision;
        return AMR_OK;
    }
    amr_status s;
    if ((s = upload(f, f->r1, f->pat.round1)) != AMR_OK) return s;
    if ((s = upload(f, f->r2, f->pat.round2)) != AMR_OK) return s;
    if ((s = upload(f, f->r1g, f->pat.round1_gather)) != AMR_OK) return s;
    if (!f->pat.round3.empty() && (s = upload(f, f->r3, f->pat.round3)) != AMR_OK) return s;
    if ((s = upload(f, f->info, f->pat.info)) != AMR_OK) return s;
    if ((s = upload(f, f->fix, f->pat.fix)) != AMR_OK) return s;
    if ((s = upload(f, f->fix_start, f->pat.fix_start)) != AMR_OK) return s;
    if ((s = upload(f, f->ranges, f->offset)) != AMR_OK) return s;
    const size_t nface = f->cfg.ndim == 3 ? size_t(f->cfg.block_n) * f->cfg.block_n : size_t(f->cfg.block_n);
    if ((s = ensure(f, f->bflux, size_t(std::max(f->pat.n_slots, 1)) * f->cfg.n_var * nface * f->esize)) != AMR_OK) return s;
    if ((s = ensure(f, f->bcdata, size_t(std::max(f->pat.n_bc, 1)) * f->cfg.n_var * nface * f->esize)) != AMR_OK) return s;
    f->pattern_rev = f->revision;
    return AMR_OK;
}

// ------------------------------------------------------------------ launches
template <class real, int D>
amr_status launch_stage(amr_forest *f, const StageArgs<real> &a, cudaStream_t st) {
    const int N = f->cfg.block_n, NG = f->cfg.n_ghost;
    if (f->cfg.physics == AMR_PHYS_ADVECTION) {
        if constexpr (std::is_same<real, float>::value) {
            // FP32 block kernel: MUSCL slopes, 8^3 / 16^3 (3D) and 8^2 .. 32^2 (2D) blocks
            if (NG == 2 && !f->scalar_stage && a.limiter <= AMR_LIM_VANLEER) {
                if (N == 8) return launch_adv_pair<D, 8>(f, a, st);
                if (N == 16) return launch_adv_pair<D, 16>(f, a, st);
                if (D == 2 && N == 32) return launch_adv_pair<D, 32>(f, a, st);
            }
        }
#define AMR_ADV_CASE(n_, g_) \
    if (N == n_ && NG == g_) return launch_stage_t<real, D, n_, g_, true, 1>(f, a, st);
        AMR_ADV_CASE(8, 2)
        AMR_ADV_CASE(16, 2)
        AMR_ADV_CASE(32, 2)
        AMR_ADV_CASE(8, 3)
        AMR_ADV_CASE(16, 3)
        AMR_ADV_CASE(32, 3)
#undef AMR_ADV_CASE
        return fail(f, AMR_EINVAL, "the advection stage needs n_ghost 2 or 3 (got %d)", NG);
    }
    if constexpr (std::is_same<real, float>::value) {
        // the pair kernels implement the MUSCL slopes with the Rusanov or HLL flux
        if (NG == 2 && !f->scalar_stage &&
            (a.limiter == AMR_LIM_MINMOD || a.limiter == AMR_LIM_MC || a.limiter == AMR_LIM_VANLEER)) {
            const bool hll = a.flux == AMR_FLUX_HLL;
            if (N == 8) return hll ? launch_stage_pair<D, 8, 1>(f, a, st) : launch_stage_pair<D, 8, 0>(f, a, st);
            if (N == 16) return hll ? launch_stage_pair<D, 16, 1>(f, a, st) : launch_stage_pair<D, 16, 0>(f, a, st);
            if (N == 32) return hll ? launch_stage_pair<D, 32, 1>(f, a, st) : launch_stage_pair<D, 32, 0>(f, a, st);
        }
    }
    const bool gen = a.limiter != AMR_LIM_MINMOD || a.flux != AMR_FLUX_RUSANOV;
#define AMR_STAGE_CASE(n_, g_)                                                                                   \
    if (N == n_ && NG == g_)                                                                                     \
        return gen ? launch_stage_t<real, D, n_, g_, true, 0>(f, a, st) : launch_stage_t<real, D, n_, g_, false, 0>(f, a, st);
    AMR_STAGE_CASE(8, 2)
    AMR_STAGE_CASE(16, 2)
    AMR_STAGE_CASE(32, 2)
    AMR_STAGE_CASE(8, 3)
    AMR_STAGE_CASE(16, 3)
    AMR_STAGE_CASE(32, 3)
#undef AMR_STAGE_CASE
    return fail(f, AMR_EINVAL, "the Euler stage needs n_ghost 2 or 3 (got %d)", NG);
}

// scratch of the WENO5 stage (face fluxes of every block); allocated
// outside stream capture
amr_status ensure_weno(amr_forest *f) {
    if (f->cfg.limiter != AMR_LIM_WENO5 || weno_fused_applies(f)) return AMR_OK;   // the single pass keeps them on chip
    const int N = f->cfg.block_n, D = f->cfg.ndim;
    const size_t nfl = size_t(D) * size_t(f->cfg.n_var) * size_t(N + 1) * size_t(D == 3 ? N * N : N);
    const size_t nb = size_t(std::max<int64_t>(nblocks(f), 1));
    return ensure(f, f->wflux, nb * nfl * size_t(f->esize));
}

template <class real, int D>
amr_status run_stage(amr_forest *f, const amr_stage *stg, cudaStream_t st) {
    StageArgs<real> a{};
    a.out = static_cast<real *>(slot_ptr(f, stg->s_out));
    a.deriv = static_cast<const real *>(slot_ptr(f, stg->s_deriv));
    a.nprev = stg->n_prev;
    for (int q = 0; q < stg->n_prev; ++q) {
        a.prev[q] = static_cast<const real *>(slot_ptr(f, stg->s_prev[q]));
        a.wprev[q] = real(stg->w_prev[q]);
    }
    a.w_dt = stg->w_dt;
    a.sc_in = static_cast<const DevScalars *>(f->sc.p);
    a.sc = static_cast<DevScalars *>(f->sc.p);
    a.info = static_cast<const BlockInfo *>(f->info.p);
    a.bflux = static_cast<real *>(f->bflux.p);
    a.update_dt = stg->update_dt;
    a.gather = stg->gather_halo;
    a.gamma = real(f->cfg.gamma);
    a.limiter = f->cfg.limiter;
    a.flux = f->cfg.flux;
    a.gravity_on = 0;
    for (int d = 0; d < 3; ++d) {
        a.grav[d] = d < D ? real(f->cfg.gravity[d]) : real(0);
        if (d < D && f->cfg.gravity[d] != 0.0) a.gravity_on = 1;
        a.vel[d] = d < D ? real(f->cfg.velocity[d]) : real(0);
    }
    amr_status s;
    if (f->cfg.limiter == AMR_LIM_WENO5) {
        // WENO5: the single-pass kernel (which may gather halos), or two
        // passes on the filled ghost cells
        if (!weno_fused_applies(f)) a.gather = 0;
        if ((s = ensure_weno(f)) != AMR_OK) return s;
        TraceSpan span(f, AMR_PHASE_STAGE, st);
        s = f->cfg.physics == AMR_PHYS_ADVECTION
                ? launch_weno<real, D, 1>(f, a, static_cast<real *>(f->wflux.p), st)
                : launch_weno<real, D, 0>(f, a, static_cast<real *>(f->wflux.p), st);
    } else {
        TraceSpan span(f, AMR_PHASE_STAGE, st);
        s = launch_stage<real, D>(f, a, st);
    }
    if (s != AMR_OK) return s;
    const int nfix = int(f->pat.fix_start.size()) - 1;
    if (nfix > 0) {
        FixArgs<real> x{};
        x.u = a.out;
        x.info = a.info;
        x.fix = static_cast<const FixFace *>(f->fix.p);
        x.fix_start = static_cast<const int32_t *>(f->fix_start.p);
        x.bflux = a.bflux;
        x.w_dt = stg->w_dt;
        x.sc = a.sc;
        x.update_dt = stg->update_dt;
        x.gamma = a.gamma;
        const int nface = D == 3 ? f->cfg.block_n * f->cfg.block_n : f->cfg.block_n;
        TraceSpan span(f, AMR_PHASE_FLUXFIX, st);
        k_fluxfix<real, D><<<nfix, std::max(32, std::min(nface, 1024)), 0, st>>>(x, f->geom);
        ++f->launches;
    }
    if (stg->update_dt) {
        TraceSpan span(f, AMR_PHASE_DT, st);
        k_dt_commit<<<(n_inst(f) + 31) / 32, 32, 0, st>>>(static_cast<DevScalars *>(f->sc.p),
                                                          static_cast<const double *>(f->cfltab.p), n_inst(f));
        ++f->launches;
    }
    CU(cudaGetLastError());
    return AMR_OK;
}

// dispatch on precision and dimension
template <template <class, int> class Fn, class... Args>
amr_status dispatch(amr_forest *f, Args &&...args) {
    if (f->cfg.precision == 64) {
        if (f->cfg.ndim == 3) return Fn<double, 3>::run(f, args...);
        return Fn<double, 2>::run(f, args...);
    }
    if (f->cfg.ndim == 3) return Fn<float, 3>::run(f, args...);
    return Fn<float, 2>::run(f, args...);
}

template <class real, int D>
struct GhostFn {
    static amr_status run(amr_forest *f, int s, cudaStream_t st, bool gather) { return launch_ghosts<real, D>(f, s, st, gather); }
};
template <class real, int D>
struct StageFn {
    static amr_status run(amr_forest *f, const amr_stage *stg, cudaStream_t st) { return run_stage<real, D>(f, stg, st); }
};
template <class real, int D>
struct MaxSpeedFn {
    static amr_status run(amr_forest *f, int s, cudaStream_t st) {
        TraceSpan span(f, AMR_PHASE_DT, st);
        if (nblocks(f) > 0) {
            k_maxspeed<real, D><<<unsigned(nblocks(f)), 256, 0, st>>>(static_cast<const real *>(slot_ptr(f, s)),
                                                                     static_cast<const BlockInfo *>(f->info.p),
                                                                     static_cast<DevScalars *>(f->sc.p), f->geom, real(f->cfg.gamma));
            ++f->launches;
        }
        k_dt_commit<<<(n_inst(f) + 31) / 32, 32, 0, st>>>(static_cast<DevScalars *>(f->sc.p),
                                                          static_cast<const double *>(f->cfltab.p), n_inst(f));
        ++f->launches;
        CU(cudaGetLastError());
        return AMR_OK;
    }
};
template <class real, int D>
struct ConservedFn {
    static amr_status run(amr_forest *f, int s, cudaStream_t st) {
        amr_status r = ensure(f, f->partial, sizeof(double) * std::max<int64_t>(nblocks(f), 1) * f->cfg.n_var);
        if (r != AMR_OK) return r;
        if ((r = ensure(f, f->sums, sizeof(double) * 8 * size_t(n_inst(f)))) != AMR_OK) return r;
        TraceSpan span(f, AMR_PHASE_CONSERVED, st);
        if (nblocks(f) > 0) {
            k_conserved_block<real, D><<<unsigned(nblocks(f)), 256, 0, st>>>(static_cast<const real *>(slot_ptr(f, s)),
                                                                            static_cast<const BlockInfo *>(f->info.p),
                                                                            static_cast<double *>(f->partial.p), f->geom);
            ++f->launches;
        }
        k_conserved_final<<<n_inst(f), 1024, 0, st>>>(static_cast<const double *>(f->partial.p),
                                                      static_cast<const int64_t *>(f->ranges.p), f->cfg.n_var,
                                                      static_cast<double *>(f->sums.p));
        ++f->launches;
        CU(cudaGetLastError());
        return AMR_OK;
    }
};
template <class real, int D>
amr_status launch_flags(amr_forest *f, int s, const amr_flag_params *p, const int32_t *list, int n, int8_t *out, cudaStream_t st) {
    const int N = f->cfg.block_n;
    const size_t smem = flags_smem(N, D);
    if (smem > 48 * 1024) CU(cudaFuncSetAttribute(k_flags<real, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    TraceSpan span(f, AMR_PHASE_FLAGS, st);
    k_flags<real, D><<<unsigned(n), unsigned(flags_threads(N)), smem, st>>>(static_cast<const real *>(slot_ptr(f, s)), f->geom,
                                                                         f->cfg.gamma, p->c_refine, p->c_derefine, p->eps,
                                                                         p->eps_abs, out, list);
    ++f->launches;
    CU(cudaGetLastError());
    return AMR_OK;
}
// The criterion: the FP32 interval screen decides the blocks whose largest
// value lies clear of both thresholds, the FP64 kernel the rest (the same
// flags as the FP64 kernel alone, bit for bit).
double screen_square(double c, double scale) { return c > 0.0 ? c * c * scale : (c == 0.0 ? 0.0 : -1.0); }
template <class real, int D>
amr_status screen_flags(amr_forest *f, int s, const amr_flag_params *p, cudaStream_t st) {
    const int64_t nb = nblocks(f);
    amr_status r = ensure(f, f->slist, sizeof(int32_t) * size_t(nb + 1));
    if (r != AMR_OK) return r;
    int32_t *cnt = static_cast<int32_t *>(f->slist.p), *list = cnt + 1;
    int8_t *out = static_cast<int8_t *>(f->flags.p);
    const real *u = static_cast<const real *>(slot_ptr(f, s));
    const int N = f->cfg.block_n;
    const size_t smem = size_t(D == 3 ? 4 : 1) * 3 * size_t(N + 2) * size_t(N + 2) * sizeof(float);
    if (smem > 48 * 1024)
        CU(cudaFuncSetAttribute(k_flags_screen<real, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    const size_t smem64 = flags_smem(N, D);
    if (smem64 > 48 * 1024) CU(cudaFuncSetAttribute(k_flags<real, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem64)));
    const double lo = 1.0 - 0x1p-40, hi = 1.0 + 0x1p-40;
    const ScreenThresholds thr{screen_square(p->c_refine, lo), screen_square(p->c_refine, hi), screen_square(p->c_derefine, lo),
                               screen_square(p->c_derefine, hi)};
    TraceSpan span(f, AMR_PHASE_FLAGS, st);
    CU(cudaMemsetAsync(cnt, 0, sizeof(int32_t), st));
    k_flags_screen<real, D><<<unsigned(nb), unsigned(flags_threads(N)), smem, st>>>(
        u, f->geom, float(f->cfg.gamma - 1.0), float(p->eps), float(p->eps_abs), thr, out, list, cnt);
    // the undecided blocks: CTAs beyond the device-side count return at once
    k_flags<real, D><<<unsigned(nb), unsigned(flags_threads(N)), smem64, st>>>(u, f->geom, f->cfg.gamma, p->c_refine,
                                                                              p->c_derefine, p->eps, p->eps_abs, out, list, cnt);
    f->launches += 2;
    CU(cudaGetLastError());
    return AMR_OK;
}
template <class real, int D>
struct FlagFn {
    static amr_status run(amr_forest *f, int s, const amr_flag_params *p, cudaStream_t st) {
        amr_status r = ensure(f, f->flags, std::max<int64_t>(nblocks(f), 1));
        if (r != AMR_OK) return r;
        if (nblocks(f) > 0) {
            return screen_flags<real, D>(f, s, p, st);
        }
        return AMR_OK;
    }
};
template <class real, int D>
struct FeatureFn {
    static amr_status run(amr_forest *f, int s, float *x, cudaStream_t st) {
        int ml = 1;
        for (const amr_config &c : f->icfg) ml = std::max(ml, c.max_level);
        if (nblocks(f) > 0) {
            const size_t smem = features_smem<real, D>(f->cfg.block_n);
            if (smem > 40 * 1024)
                CU(cudaFuncSetAttribute(k_features<real, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            TraceSpan span(f, AMR_PHASE_FLAGS, st);
            k_features<real, D><<<unsigned(nblocks(f)), 256, smem, st>>>(static_cast<const real *>(slot_ptr(f, s)),
                                                                    static_cast<const BlockInfo *>(f->info.p), f->geom,
                                                                    f->cfg.gamma, 1.0f / float(ml), x, nblocks(f));
            ++f->launches;
        }
        CU(cudaGetLastError());
        return AMR_OK;
    }
};
template <class real, int D>
struct ListFlagFn {
    static amr_status run(amr_forest *f, int s, const amr_flag_params *p, const int32_t *list, int n, int8_t *out, cudaStream_t st) {
        if (n > 0) {
            return launch_flags<real, D>(f, s, p, list, n, out, st);
        }
        return AMR_OK;
    }
};
template <class real, int D>
struct TransferFn {
    static amr_status run(amr_forest *f, const void *uold, int n_new, cudaStream_t st) {
        if (n_new > 0) {
            k_transfer<real, D><<<unsigned(n_new), 256, 0, st>>>(static_cast<const real *>(uold), static_cast<real *>(slot_ptr(f, 0)),
                                                                static_cast<const TransferOp *>(f->ops.p), f->geom);
            ++f->launches;
        }
        CU(cudaGetLastError());
        return AMR_OK;
    }
};

// One time step as a sequence of Eq. 5 sub-steps, each preceded by the ghost
// fill of the slot it differentiates; the last one updates dt.
//   Heun (Eq. 6-7):  u1 = u0 + dt L(u0);  u0' = (u0 + u1 + dt L(u1)) / 2
//   SSP3 (Shu-Osher): u1 = u0 + dt L(u0);  u2 = 3/4 u0 + 1/4 (u1 + dt L(u1));
//                    u0' = 1/3 u0 + 2/3 (u2 + dt L(u2))
//   SSP43 (four stages, third order): u1 = u0 + dt/2 L(u0);
//        u2 = u1 + dt/2 L(u1);  u3 = 2/3 u0 + 1/3 u2 + dt/6 L(u2);
//        u0' = u3 + dt/2 L(u3)   (u3 stored in slot 1)
//   RK4: u1 = u0 + dt/2 L(u0);  u2 = u0 + dt/2 L(u1);  u3 = u0 + dt L(u2);
//        u0' = u0 + dt/6 (k1 + 2 k2 + 2 k3 + k4) with k1 = 2 (u1 - u0) / dt,
//        k2 = 2 (u2 - u0) / dt, k3 = (u3 - u0) / dt, k4 = L(u3), i.e.
//        u0' = -1/3 u0 + 1/3 u1 + 2/3 u2 + 1/3 u3 + dt/6 L(u3)
int step_slots(int flags) { return (flags & AMR_STEP_RK4) ? 4 : ((flags & (AMR_STEP_SSP3 | AMR_STEP_SSP43)) ? 3 : 2); }

amr_status rk_step(amr_forest *f, cudaStream_t st, bool gather, int flags) {
    if (f->cfg.limiter == AMR_LIM_WENO5 && !weno_fused_applies(f)) gather = false;   // the two-pass form reads filled ghosts
    const int gh = gather ? 1 : 0;
    std::vector<amr_stage> seq;
    if (flags & AMR_STEP_RK4) {
        seq.push_back({1, 0, 1, {0, 0, 0, 0}, {1.0, 0, 0, 0}, 0.5, 0, gh});
        seq.push_back({2, 1, 1, {0, 0, 0, 0}, {1.0, 0, 0, 0}, 0.5, 0, gh});
        seq.push_back({3, 2, 1, {0, 0, 0, 0}, {1.0, 0, 0, 0}, 1.0, 0, gh});
        seq.push_back({0, 3, 4, {0, 1, 2, 3}, {-1.0 / 3.0, 1.0 / 3.0, 2.0 / 3.0, 1.0 / 3.0}, 1.0 / 6.0, 1, gh});
    } else if (flags & AMR_STEP_SSP43) {
        seq.push_back({1, 0, 1, {0, 0, 0, 0}, {1.0, 0, 0, 0}, 0.5, 0, gh});
        seq.push_back({2, 1, 1, {1, 0, 0, 0}, {1.0, 0, 0, 0}, 0.5, 0, gh});
        seq.push_back({1, 2, 2, {0, 2, 0, 0}, {2.0 / 3.0, 1.0 / 3.0, 0, 0}, 1.0 / 6.0, 0, gh});
        seq.push_back({0, 1, 1, {1, 0, 0, 0}, {1.0, 0, 0, 0}, 0.5, 1, gh});
    } else if (flags & AMR_STEP_SSP3) {
        seq.push_back({1, 0, 1, {0, 0, 0, 0}, {1.0, 0, 0, 0}, 1.0, 0, gh});
        seq.push_back({2, 1, 2, {0, 1, 0, 0}, {0.75, 0.25, 0, 0}, 0.25, 0, gh});
        seq.push_back({0, 2, 2, {0, 2, 0, 0}, {1.0 / 3.0, 2.0 / 3.0, 0, 0}, 2.0 / 3.0, 1, gh});
    } else {
        seq.push_back({1, 0, 1, {0, 0, 0, 0}, {1.0, 0, 0, 0}, 1.0, 0, gh});
        seq.push_back({0, 1, 2, {0, 1, 0, 0}, {0.5, 0.5, 0, 0}, 0.5, 1, gh});
    }
    amr_status r;
    for (const amr_stage &s : seq) {
        if ((r = dispatch<GhostFn>(f, s.s_deriv, st, gather)) != AMR_OK) return r;
        if ((r = dispatch<StageFn>(f, &s, st)) != AMR_OK) return r;
    }
    return AMR_OK;
}

bool valid_slot(const amr_forest *f, int s) { return s >= 0 && s < f->cfg.n_states; }

#define NEED_DEVICE(f) \
    do {               \
        if ((f)->cfg.host_only) return fail(f, AMR_ESTATE, "host-only forest has no block data"); \
    } while (0)

}  // namespace

// =================================================================== C ABI
extern "C" {

amr_status amr_create_batch(const amr_config *cfgs, const int *init_levels, int n, amr_forest **out) {
    if (!cfgs || !init_levels || !out || n < 1) return AMR_EINVAL;
    *out = nullptr;
    std::string why;
    int64_t capacity = 0;
    for (int i = 0; i < n; ++i) {
        const amr_config &c = cfgs[i], &c0 = cfgs[0];
        if (validate(&c, why) != AMR_OK) return AMR_EINVAL;
        if (init_levels[i] < 0 || init_levels[i] > c.max_level) return AMR_EINVAL;
        // settings every instance of one forest shares
        if (c.ndim != c0.ndim || c.block_n != c0.block_n || c.n_ghost != c0.n_ghost || c.precision != c0.precision ||
            c.n_states != c0.n_states || c.gamma != c0.gamma || c.host_only != c0.host_only ||
            c.limiter != c0.limiter || c.flux != c0.flux || c.gravity[0] != c0.gravity[0] ||
            c.gravity[1] != c0.gravity[1] || c.gravity[2] != c0.gravity[2] || c.diagonal_ghosts != c0.diagonal_ghosts ||
            c.physics != c0.physics || c.velocity[0] != c0.velocity[0] || c.velocity[1] != c0.velocity[1] ||
            c.velocity[2] != c0.velocity[2] ||
            c.dev_alloc != c0.dev_alloc || c.dev_free != c0.dev_free || c.alloc_ctx != c0.alloc_ctx)
            return AMR_EINVAL;
        capacity += c.max_blocks;
    }
    if (capacity > (int64_t(1) << 31) - 1) return AMR_EINVAL;
    amr_forest *f = new (std::nothrow) amr_forest();
    if (!f) return AMR_ENOMEM;
    f->cfg = cfgs[0];
    f->cfg.max_blocks = int(capacity);
    f->icfg.assign(cfgs, cfgs + n);
    f->esize = f->cfg.precision / 8;
    if (!f->cfg.host_only) {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&f->n_sms, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
    }
    fill_geom(f);
    f->block_bytes = size_t(f->geom.bstride) * f->esize;
    f->inst.resize(size_t(n));
    for (int i = 0; i < n; ++i) {
        const amr_config &c = cfgs[i];
        Geometry G;
        G.ndim = c.ndim;
        for (int d = 0; d < 3; ++d) {
            G.ntrees[d] = d < c.ndim ? c.ntrees[d] : 1;
            G.periodic[d] = d < c.ndim ? (c.periodic[d] ? 1 : 0) : 1;
        }
        G.max_level = c.max_level;
        int64_t n0 = 1;
        for (int d = 0; d < c.ndim; ++d) n0 *= G.extent(d, init_levels[i]);
        if (n0 > c.max_blocks) {
            delete f;
            return AMR_ECAPACITY;
        }
        f->inst[size_t(i)].init_uniform(G, init_levels[i]);
    }
    set_offsets(f);
    if (f->cfg.host_only) {
        amr_status s = upload_pattern(f);
        if (s != AMR_OK) {
            delete f;
            return s;
        }
        *out = f;
        return AMR_OK;
    }
    const size_t bytes = size_t(f->cfg.n_states) * size_t(capacity) * f->block_bytes;
    f->state = dev_alloc(f, bytes);
    amr_status s = AMR_OK;
    if (!f->state) s = AMR_ENOMEM;
    if (s == AMR_OK && cudaMemset(f->state, 0, bytes) != cudaSuccess) s = AMR_ECUDA;
    if (s == AMR_OK) s = ensure(f, f->sc, sizeof(DevScalars) * size_t(n));
    if (s == AMR_OK && cudaMemset(f->sc.p, 0, sizeof(DevScalars) * size_t(n)) != cudaSuccess) s = AMR_ECUDA;
    if (s == AMR_OK) s = upload_tables(f);
    if (s == AMR_OK) s = upload_pattern(f);
    if (s == AMR_OK && cudaStreamCreateWithFlags(&f->cap_stream, cudaStreamNonBlocking) != cudaSuccess) s = AMR_ECUDA;
    if (s != AMR_OK) {
        cudaGetLastError();
        amr_destroy_forest(f);
        return s;
    }
    *out = f;
    return AMR_OK;
}

amr_status amr_create_forest(const amr_config *cfg, int init_level, amr_forest **out) {
    return amr_create_batch(cfg, &init_level, 1, out);
}

amr_status amr_n_instances(const amr_forest *f, int *n) {
    if (!f || !n) return AMR_EINVAL;
    *n = n_inst(f);
    return AMR_OK;
}

amr_status amr_instance_blocks(const amr_forest *f, int inst, int64_t *first, int64_t *n) {
    if (!f || inst < 0 || inst >= n_inst(f)) return AMR_EINVAL;
    if (first) *first = f->offset[size_t(inst)];
    if (n) *n = f->offset[size_t(inst) + 1] - f->offset[size_t(inst)];
    return AMR_OK;
}

amr_status amr_destroy_forest(amr_forest *f) {
    if (!f) return AMR_OK;
    if (f->gexec) cudaGraphExecDestroy(f->gexec);
    if (f->cap_stream) cudaStreamDestroy(f->cap_stream);
    for (DBuf *b : {&f->r1, &f->r2, &f->r1g, &f->r3, &f->info, &f->fix, &f->fix_start, &f->bflux, &f->bcdata, &f->sc, &f->partial, &f->sums,
                    &f->flags, &f->ops, &f->level, &f->dxtab, &f->invdxtab, &f->bctype, &f->bcval, &f->cfltab, &f->ranges,
                    &f->feat, &f->prob, &f->mflags, &f->flist, &f->slist, &f->wflux})
        dev_free(f, b->p);
    dev_free(f, f->state);
    for (const TraceRec &t : f->trace_open) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : f->ev_free) cudaEventDestroy(e);
    delete f;
    return AMR_OK;
}

amr_status amr_n_blocks(const amr_forest *f, int64_t *n) {
    if (!f || !n) return AMR_EINVAL;
    *n = nblocks(f);
    return AMR_OK;
}

amr_status amr_get_blocks(const amr_forest *f, int32_t *level, int64_t *coords, int64_t cap, int64_t *n) {
    if (!f || cap < 0) return AMR_EINVAL;
    const int64_t nb = nblocks(f);
    if (n) *n = nb;
    for (int64_t b = 0; b < std::min(cap, nb); ++b) {
        const Leaf &l = leaf_at(f, b);
        if (level) level[b] = l.lev;
        if (coords)
            for (int d = 0; d < 3; ++d) coords[3 * b + d] = d < f->cfg.ndim ? l.g[d] : 0;
    }
    return AMR_OK;
}

amr_status amr_build_ghost_pattern(amr_forest *f) {
    if (!f) return AMR_EINVAL;
    return upload_pattern(f);
}

amr_status amr_get_ghost_pattern(const amr_forest *f, amr_ghost_entry *out, int64_t cap, int64_t *n) {
    if (!f || cap < 0 || (cap > 0 && !out)) return AMR_EINVAL;
    if (f->pattern_rev != f->revision) return AMR_ESTATE;
    const auto &e = f->pat.entries;
    if (n) *n = int64_t(e.size());
    for (int64_t i = 0; i < std::min<int64_t>(cap, int64_t(e.size())); ++i)
        out[i] = {e[i].kind, e[i].face, e[i].dst, e[i].src, e[i].offset, e[i].aux};
    return AMR_OK;
}

amr_status amr_set_state(amr_forest *f, int s, const void *src, int on_device, amr_stream stream) {
    if (!f || !src || !valid_slot(f, s)) return AMR_EINVAL;
    NEED_DEVICE(f);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = size_t(nblocks(f)) * f->block_bytes;
    CU(cudaMemcpyAsync(slot_ptr(f, s), src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (!on_device) CU(cudaStreamSynchronize(st));
    return AMR_OK;
}

amr_status amr_get_state(const amr_forest *fc, int s, void *dst, int on_device, amr_stream stream) {
    amr_forest *f = const_cast<amr_forest *>(fc);
    if (!f || !dst || !valid_slot(f, s)) return AMR_EINVAL;
    NEED_DEVICE(f);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = size_t(nblocks(f)) * f->block_bytes;
    CU(cudaMemcpyAsync(dst, slot_ptr(f, s), bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (!on_device) CU(cudaStreamSynchronize(st));
    return AMR_OK;
}

amr_status amr_state_ptr(const amr_forest *f, int s, void **ptr) {
    if (!f || !ptr || !valid_slot(f, s)) return AMR_EINVAL;
    if (f->cfg.host_only) return AMR_ESTATE;
    *ptr = slot_ptr(f, s);
    return AMR_OK;
}

amr_status amr_set_bc_data(amr_forest *f, const double *values, int64_t n_values) {
    if (!f || (n_values > 0 && !values)) return AMR_EINVAL;
    NEED_DEVICE(f);
    amr_status r = upload_pattern(f);
    if (r != AMR_OK) return r;
    const int64_t nface = f->cfg.ndim == 3 ? int64_t(f->cfg.block_n) * f->cfg.block_n : f->cfg.block_n;
    const int64_t need = int64_t(f->pat.n_bc) * f->cfg.n_var * nface;
    if (n_values != need) return fail(f, AMR_EINVAL, "bc_data needs %lld values, got %lld", (long long)need, (long long)n_values);
    if (need == 0) return AMR_OK;
    if (f->cfg.precision == 64) {
        CU(cudaMemcpy(f->bcdata.p, values, sizeof(double) * need, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> tmp(values, values + need);
        CU(cudaMemcpy(f->bcdata.p, tmp.data(), sizeof(float) * need, cudaMemcpyHostToDevice));
    }
    return AMR_OK;
}

amr_status amr_fill_ghosts(amr_forest *f, int s, amr_stream stream) {
    if (!f || !valid_slot(f, s)) return AMR_EINVAL;
    NEED_DEVICE(f);
    amr_status r = upload_pattern(f);
    if (r != AMR_OK) return r;
    return dispatch<GhostFn>(f, s, static_cast<cudaStream_t>(stream), false);
}

amr_status amr_compute_dt(amr_forest *f, int s, amr_stream stream) {
    if (!f || !valid_slot(f, s)) return AMR_EINVAL;
    NEED_DEVICE(f);
    return dispatch<MaxSpeedFn>(f, s, static_cast<cudaStream_t>(stream));
}

amr_status amr_set_dt(amr_forest *f, double dt, amr_stream stream) {
    if (!f || !(dt >= 0.0)) return AMR_EINVAL;
    NEED_DEVICE(f);
    // every instance's dt (the first field of each DevScalars)
    std::vector<double> v(size_t(n_inst(f)), dt);
    CU(cudaMemcpy2DAsync(f->sc.p, sizeof(DevScalars), v.data(), sizeof(double), sizeof(double), v.size(),
                         cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream)));
    CU(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return AMR_OK;
}

amr_status amr_get_dts(amr_forest *f, double *dts, amr_stream stream) {
    if (!f || !dts) return AMR_EINVAL;
    NEED_DEVICE(f);
    CU(cudaMemcpy2DAsync(dts, sizeof(double), f->sc.p, sizeof(DevScalars), sizeof(double), size_t(n_inst(f)),
                         cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)));
    CU(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return AMR_OK;
}

amr_status amr_get_dt(amr_forest *f, double *dt, amr_stream stream) {
    if (!f || !dt) return AMR_EINVAL;
    NEED_DEVICE(f);
    CU(cudaMemcpyAsync(dt, f->sc.p, sizeof(double), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)));
    CU(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return AMR_OK;
}

amr_status amr_advance_stage(amr_forest *f, const amr_stage *st, amr_stream stream) {
    if (!f || !st) return AMR_EINVAL;
    NEED_DEVICE(f);
    if (!valid_slot(f, st->s_out) || !valid_slot(f, st->s_deriv) || st->n_prev < 0 || st->n_prev > 4) return AMR_EINVAL;
    for (int q = 0; q < st->n_prev; ++q)
        if (!valid_slot(f, st->s_prev[q])) return AMR_EINVAL;
    if (st->s_out == st->s_deriv) return fail(f, AMR_EINVAL, "s_out must differ from s_deriv");
    if (f->cfg.n_ghost < 2) return fail(f, AMR_EINVAL, "the Euler stage needs n_ghost >= 2");
    amr_status r = upload_pattern(f);
    if (r != AMR_OK) return r;
    return dispatch<StageFn>(f, st, static_cast<cudaStream_t>(stream));
}

amr_status amr_step(amr_forest *f, int n_steps, int flags, amr_stream stream) {
    if (!f || n_steps < 0) return AMR_EINVAL;
    NEED_DEVICE(f);
    const int schemes = flags & (AMR_STEP_SSP3 | AMR_STEP_RK4 | AMR_STEP_SSP43);
    if (schemes & (schemes - 1)) return fail(f, AMR_EINVAL, "choose one Runge-Kutta scheme");
    if (f->cfg.n_states < step_slots(flags))
        return fail(f, AMR_EINVAL, "this Runge-Kutta scheme needs n_states >= %d", step_slots(flags));
    if (f->cfg.n_ghost < 2) return fail(f, AMR_EINVAL, "the Euler stage needs n_ghost >= 2");
    amr_status r = upload_pattern(f);
    if (r != AMR_OK) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool gather = (flags & AMR_STEP_GATHER) != 0;
    if (!(flags & AMR_STEP_GRAPH) || f->tracing) {
        for (int i = 0; i < n_steps; ++i)
            if ((r = rk_step(f, st, gather, flags)) != AMR_OK) return r;
        return AMR_OK;
    }
    if (!f->gexec || f->graph_rev != f->revision || f->graph_flags != flags) {
        if (f->gexec) {
            cudaGraphExecDestroy(f->gexec);
            f->gexec = nullptr;
        }
        // capture one step on the library's own stream, after the caller's
        // stream has drained (capture needs a non-legacy stream); buffers
        // are allocated before the capture
        if ((r = ensure_weno(f)) != AMR_OK) return r;
        CU(cudaStreamSynchronize(st));
        const int64_t before = f->launches;
        CU(cudaStreamBeginCapture(f->cap_stream, cudaStreamCaptureModeThreadLocal));
        r = rk_step(f, f->cap_stream, gather, flags);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(f->cap_stream, &graph);
        if (r != AMR_OK) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e != cudaSuccess) return fail(f, AMR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        f->graph_nodes = f->launches - before;
        f->launches = before;
        e = cudaGraphInstantiate(&f->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(f, AMR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        f->graph_rev = f->revision;
        f->graph_flags = flags;
    }
    for (int i = 0; i < n_steps; ++i) {
        CU(cudaGraphLaunch(f->gexec, st));
        f->launches += f->graph_nodes;
    }
    return AMR_OK;
}

amr_status amr_conserved(amr_forest *f, int s, double *sums, amr_stream stream) {
    if (!f || !sums || !valid_slot(f, s)) return AMR_EINVAL;
    NEED_DEVICE(f);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    amr_status r = dispatch<ConservedFn>(f, s, st);
    if (r != AMR_OK) return r;
    CU(cudaMemcpyAsync(sums, f->sums.p, sizeof(double) * f->cfg.n_var, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return AMR_OK;
}

amr_status amr_conserved_all(amr_forest *f, int s, double *sums, amr_stream stream) {
    if (!f || !sums || !valid_slot(f, s)) return AMR_EINVAL;
    NEED_DEVICE(f);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    amr_status r = dispatch<ConservedFn>(f, s, st);
    if (r != AMR_OK) return r;
    CU(cudaMemcpyAsync(sums, f->sums.p, sizeof(double) * f->cfg.n_var * size_t(n_inst(f)), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return AMR_OK;
}

amr_status amr_flag(amr_forest *f, int s, const amr_flag_params *p, int8_t *flags_out, amr_stream stream) {
    if (!f || !p || !flags_out || !valid_slot(f, s)) return AMR_EINVAL;
    NEED_DEVICE(f);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    amr_status r = dispatch<FlagFn>(f, s, p, st);
    if (r != AMR_OK) return r;
    if (nblocks(f) > 0) CU(cudaMemcpyAsync(flags_out, f->flags.p, size_t(nblocks(f)), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return AMR_OK;
}

amr_status amr_flag_and_regrid(amr_forest *f, const amr_flag_params *p, const int8_t *flags, int *changed, amr_stream stream) {
    if (!f || (!flags && !p)) return AMR_EINVAL;
    if (changed) *changed = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    amr_status r = AMR_OK;
    const int64_t nb = nblocks(f);
    const int ni = n_inst(f);
    std::vector<int8_t> fl(size_t(std::max<int64_t>(nb, 1)));
    if (f->cfg.host_only) {
        if (!flags) return fail(f, AMR_ESTATE, "host-only forest: regrid needs explicit flags");
        std::copy(flags, flags + nb, fl.begin());
    } else {
        r = amr_fill_ghosts(f, 0, stream);
        if (r != AMR_OK) return r;
        if (flags) std::copy(flags, flags + nb, fl.begin());
        else if ((r = amr_flag(f, 0, p, fl.data(), stream)) != AMR_OK) return r;
    }
    // adapt every instance with its slice of the flags (Sec. 2.2)
    std::unique_ptr<HostSpan> mesh_span(new HostSpan(f, AMR_PHASE_MESH_HOST));
    std::vector<std::vector<Leaf>> nl(static_cast<size_t>(ni));
    std::vector<char> moved(size_t(ni), 0);
    int64_t total = 0;
    bool any = false;
    for (int i = 0; i < ni; ++i) {
        const Forest &F = f->inst[size_t(i)];
        std::vector<int8_t> part(fl.begin() + f->offset[size_t(i)], fl.begin() + f->offset[size_t(i) + 1]);
        nl[size_t(i)] = F.adapted(part);
        bool same = nl[size_t(i)].size() == F.leaves.size();
        for (size_t k = 0; same && k < nl[size_t(i)].size(); ++k) same = pack_key(nl[size_t(i)][k]) == pack_key(F.leaves[k]);
        moved[size_t(i)] = !same;
        any = any || !same;
        total += int64_t(nl[size_t(i)].size());
        if (int64_t(nl[size_t(i)].size()) > f->icfg[size_t(i)].max_blocks)
            return fail(f, AMR_ECAPACITY, "regrid of instance %d needs %zu blocks, its capacity is %d", i, nl[size_t(i)].size(),
                        f->icfg[size_t(i)].max_blocks);
    }
    if (!any) return AMR_OK;
    if (total > f->cfg.max_blocks) return fail(f, AMR_ECAPACITY, "regrid needs %lld blocks, capacity is %d", (long long)total, f->cfg.max_blocks);
    if (f->cfg.host_only) {
        for (int i = 0; i < ni; ++i)
            if (moved[size_t(i)]) f->inst[size_t(i)].assign(std::move(nl[size_t(i)]));
        set_offsets(f);
        ++f->revision;
        mesh_span.reset();
        if ((r = upload_pattern(f)) != AMR_OK) return r;
        if (changed) *changed = 1;
        return AMR_OK;
    }
    // old -> new map (Sec. 2.2: copied, refined and coarsened blocks); block
    // indices are global (instance offset + local)
    const int D = f->cfg.ndim;
    std::vector<TransferOp> ops;
    ops.reserve(size_t(total));
    for (int i = 0; i < ni; ++i) {
        const Forest &F = f->inst[size_t(i)];
        const int o0 = int(f->offset[size_t(i)]);
        for (size_t b = 0; b < nl[size_t(i)].size(); ++b) {
            const Leaf &l = nl[size_t(i)][b];
            TransferOp op{};
            int o = F.find(l.lev, l.g[0], l.g[1], l.g[2]);
            if (o >= 0) {
                op.kind = 0;
                op.src[0] = o0 + o;
            } else if (l.lev > 0 && (o = F.find(l.lev - 1, l.g[0] >> 1, l.g[1] >> 1, D == 3 ? l.g[2] >> 1 : 0)) >= 0) {
                op.kind = 1;
                op.src[0] = o0 + o;
                op.pos = int(l.g[0] & 1) | int(l.g[1] & 1) << 1 | (D == 3 ? int(l.g[2] & 1) << 2 : 0);
            } else {
                op.kind = 2;
                for (int c = 0; c < (1 << D); ++c) {
                    int sidx = F.find(l.lev + 1, 2 * l.g[0] + (c & 1), 2 * l.g[1] + ((c >> 1) & 1),
                                      D == 3 ? 2 * l.g[2] + ((c >> 2) & 1) : 0);
                    if (sidx < 0) return fail(f, AMR_ESTATE, "regrid: a block of instance %d changed by more than one level", i);
                    op.src[c] = o0 + sidx;
                }
            }
            ops.push_back(op);
        }
    }
    mesh_span.reset();
    // temporary copy of the old blocks (slot 1 when available)
    void *tmp = nullptr;
    bool own_tmp = false;
    const size_t old_bytes = size_t(nb) * f->block_bytes;
    if (f->cfg.n_states >= 2) {
        tmp = slot_ptr(f, 1);
    } else {
        tmp = dev_alloc(f, old_bytes);
        if (!tmp) return fail(f, AMR_ENOMEM, "regrid: no room for the old blocks");
        own_tmp = true;
    }
    if ((r = upload(f, f->ops, ops)) != AMR_OK) return r;
    {
        TraceSpan span(f, AMR_PHASE_TRANSFER, st);
        CU(cudaMemcpyAsync(tmp, slot_ptr(f, 0), old_bytes, cudaMemcpyDeviceToDevice, st));
        r = dispatch<TransferFn>(f, static_cast<const void *>(tmp), int(total), st);
    }
    if (own_tmp) {
        cudaStreamSynchronize(st);
        dev_free(f, tmp);
    }
    if (r != AMR_OK) return r;
    for (int i = 0; i < ni; ++i)
        if (moved[size_t(i)]) f->inst[size_t(i)].assign(std::move(nl[size_t(i)]));
    set_offsets(f);
    ++f->revision;
    if ((r = upload_pattern(f)) != AMR_OK) return r;
    // the time step of the new mesh: the CFL limit of slot 0 (Sec. 3.2) --
    // refined blocks have smaller cells than the ones the last stage saw
    if ((r = dispatch<MaxSpeedFn>(f, 0, st)) != AMR_OK) return r;
    CU(cudaStreamSynchronize(st));
    if (changed) *changed = 1;
    return AMR_OK;
}

amr_status amr_sync_status(amr_forest *f, amr_stream stream) {
    if (!f) return AMR_EINVAL;
    NEED_DEVICE(f);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevScalars h{};
    CU(cudaMemcpyAsync(&h, f->sc.p, sizeof h, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (h.status != 0) {
        const int zero = 0;
        CU(cudaMemcpy(static_cast<char *>(f->sc.p) + offsetof(DevScalars, status), &zero, sizeof zero, cudaMemcpyHostToDevice));
        return fail(f, amr_status(h.status), "device reported status %d", h.status);
    }
    return AMR_OK;
}

amr_status amr_features(amr_forest *f, int s, float *x, int *n_features, amr_stream stream) {
    if (!f || !valid_slot(f, s)) return AMR_EINVAL;
    NEED_DEVICE(f);
    if (f->cfg.block_n % 4) return fail(f, AMR_EINVAL, "features pool 4 cells per dimension: block_n must be a multiple of 4");
    if (f->cfg.physics != AMR_PHYS_EULER) return fail(f, AMR_EINVAL, "the flag features are Euler quantities (density, pressure, speed)");
    const int F = 3 * (f->cfg.ndim == 3 ? 64 : 16) + 1;
    if (n_features) *n_features = F;
    if (!x) return AMR_OK;
    amr_status r = upload_pattern(f);
    if (r != AMR_OK) return r;
    return dispatch<FeatureFn>(f, s, x, static_cast<cudaStream_t>(stream));
}

amr_status amr_mlp_flags(amr_forest *f, amr_mlp *m, int s, const amr_flag_params *p, double tau, int8_t *flags_out,
                         int64_t *n_fallback, amr_stream stream) {
    if (!f || !m || !p || !flags_out || !valid_slot(f, s)) return AMR_EINVAL;
    NEED_DEVICE(f);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int F = 0;
    amr_status r = amr_features(f, s, nullptr, &F, stream);
    if (r != AMR_OK) return r;
    if (F != m->F) return fail(f, AMR_EINVAL, "the model takes %d features, this forest gives %d", m->F, F);
    const int64_t nb = nblocks(f);
    if (nb == 0) return AMR_OK;
    if ((r = ensure(f, f->feat, sizeof(float) * size_t(F) * size_t(nb))) != AMR_OK) return r;
    if ((r = ensure(f, f->prob, sizeof(float) * 3 * size_t(nb))) != AMR_OK) return r;
    if ((r = ensure(f, f->mflags, size_t(nb))) != AMR_OK) return r;
    if ((r = amr_features(f, s, static_cast<float *>(f->feat.p), nullptr, stream)) != AMR_OK) return r;
    if ((r = amr_mlp_forward(m, static_cast<const float *>(f->feat.p), nb, static_cast<float *>(f->prob.p), stream)) != AMR_OK)
        return fail(f, r, "model forward pass failed");
    k_mlp_decide<<<unsigned((nb + 255) / 256), 256, 0, st>>>(static_cast<const float *>(f->prob.p), nb, float(tau),
                                                             static_cast<int8_t *>(f->mflags.p));
    f->launches += 2;
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(flags_out, f->mflags.p, size_t(nb), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    // low-confidence blocks fall back to the criterion of Eq. 12
    std::vector<int32_t> list;
    for (int64_t b = 0; b < nb; ++b)
        if (flags_out[b] == 2) list.push_back(int32_t(b));
    if (n_fallback) *n_fallback = int64_t(list.size());
    if (list.empty()) return AMR_OK;
    if ((r = amr_fill_ghosts(f, s, stream)) != AMR_OK) return r;
    if ((r = upload(f, f->flist, list)) != AMR_OK) return r;
    if ((r = dispatch<ListFlagFn>(f, s, p, static_cast<const int32_t *>(f->flist.p), int(list.size()),
                                  static_cast<int8_t *>(f->mflags.p), st)) != AMR_OK)
        return r;
    CU(cudaMemcpyAsync(flags_out, f->mflags.p, size_t(nb), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return AMR_OK;
}

amr_status amr_autotune(amr_forest *f, int *choice, double *best_ms, amr_stream stream) {
    if (!f) return AMR_EINVAL;
    NEED_DEVICE(f);
    if (f->cfg.n_states < 2 || f->cfg.n_ghost < 2) return fail(f, AMR_EINVAL, "autotuning times a stage into slot 1 (needs n_states >= 2, n_ghost >= 2)");
    amr_status r = upload_pattern(f);
    if (r != AMR_OK) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the candidates' timings are not phases of a step: tracing pauses
    struct Pause {
        amr_forest *f;
        bool was;
        ~Pause() { f->tracing = was; }
    } pause{f, f->tracing};
    f->tracing = false;
    // candidates: blocks (tiles) per CTA 1, 2, 4 or a persistent grid, for
    // each kernel / staging tile: the FP32 pair kernel (2D or 3D) with tile
    // 16 and, for blocks above 8 cells a side, tile 8, or the FP32 advection
    // block kernel; the per-cell kernel
    struct Cand { bool scalar; int ipc; bool pers; int tile; };
    std::vector<Cand> cands;
    const bool pair_ok = f->cfg.precision == 32 && f->cfg.n_ghost == 2 && f->cfg.limiter <= AMR_LIM_VANLEER &&
                         f->cfg.physics == AMR_PHYS_EULER;
    // the FP32 advection block kernel (any flux: both are upwind)
    const bool adv_ok = f->cfg.precision == 32 && f->cfg.n_ghost == 2 && f->cfg.limiter <= AMR_LIM_VANLEER &&
                        f->cfg.physics == AMR_PHYS_ADVECTION &&
                        (f->cfg.block_n <= 16 || (f->cfg.ndim == 2 && f->cfg.block_n == 32));
    std::vector<std::pair<bool, int>> kernels;   // (per-cell kernel, pair tile)
    if (pair_ok) {
        kernels.push_back({false, 0});
        if (f->cfg.block_n > 8) kernels.push_back({false, 8});
    }
    if (adv_ok) kernels.push_back({false, 0});
    kernels.push_back({true, 0});
    for (const auto &k : kernels) {
        for (int ipc : {1, 2, 4}) cands.push_back({k.first, ipc, false, k.second});
        cands.push_back({k.first, 1, true, k.second});
    }
    // a stage that leaves slot 0 alone: slot 1 = slot 0 (w_dt = 0), halos gathered
    amr_stage probe{1, 0, 1, {0, 0, 0, 0}, {1.0, 0, 0, 0}, 0.0, 0, 1};
    if ((r = dispatch<GhostFn>(f, 0, st, true)) != AMR_OK) return r;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    int best = -1;
    float best_t = 0.f;
    for (size_t c = 0; c < cands.size(); ++c) {
        f->scalar_stage = cands[c].scalar;
        f->items_per_cta = cands[c].ipc;
        f->persistent = cands[c].pers;
        f->pair_tile = cands[c].tile;
        if ((r = dispatch<StageFn>(f, &probe, st)) != AMR_OK) break;      // warm-up
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 3; ++rep)
            if ((r = dispatch<StageFn>(f, &probe, st)) != AMR_OK) break;
        cudaEventRecord(e1, st);
        if (r != AMR_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { r = AMR_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        if (best < 0 || ms < best_t) { best = int(c); best_t = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != AMR_OK) return r;
    f->scalar_stage = cands[size_t(best)].scalar;
    f->items_per_cta = cands[size_t(best)].ipc;
    f->persistent = cands[size_t(best)].pers;
    f->pair_tile = cands[size_t(best)].tile;
    f->graph_rev = ~0ull;     // launch shapes changed: re-capture
    if (choice)
        *choice = (f->scalar_stage ? 100 : 0) + (f->pair_tile == 8 ? 1000 : 0) + (f->persistent ? 0 : f->items_per_cta);
    if (best_ms) *best_ms = best_t;
    return AMR_OK;
}

amr_status amr_set_launch_shape(amr_forest *f, int choice) {
    if (!f || choice < 0) return AMR_EINVAL;
    const int tile8 = choice / 1000, scalar = (choice % 1000) / 100, ipc = choice % 100;
    if (tile8 > 1 || scalar > 1 || ipc > 64 || (tile8 && scalar)) return AMR_EINVAL;
    const bool pair_ok = f->cfg.precision == 32 && f->cfg.n_ghost == 2 && f->cfg.limiter <= AMR_LIM_VANLEER &&
                         f->cfg.physics == AMR_PHYS_EULER;
    if (tile8 && (!pair_ok || f->cfg.block_n <= 8)) return fail(f, AMR_EINVAL, "8 x 8 tiles need an FP32 pair kernel and blocks above 8 cells a side");
    f->scalar_stage = scalar == 1;
    f->pair_tile = tile8 ? 8 : 0;
    f->persistent = ipc == 0;
    f->items_per_cta = ipc == 0 ? 1 : ipc;
    f->graph_rev = ~0ull;
    return AMR_OK;
}

}  // extern "C"

// ------------------------------------------------------ checkpoint and output
namespace {

constexpr char kCkptMagic[8] = {'A', 'M', 'R', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 2;

struct CkptHead {
    char magic[8];
    uint32_t version, n_inst;
    int32_t precision, ndim, block_n, n_ghost, n_var, n_states, host_only, limiter, flux, diagonal_ghosts;
    double gamma, gravity[3];
    int32_t physics, pad;
    double velocity[3];
    int64_t n_blocks;
};
struct CkptInst {
    int32_t ntrees[3], periodic[3], max_level, max_blocks, bc[6];
    double lo[3], len[3], cfl, bc_val[6][8], dt;
    int64_t n_leaves;
};
struct CkptLeaf {
    int32_t lev, pad;
    int64_t g[3];
};

struct CFile {
    FILE *fp = nullptr;
    ~CFile() {
        if (fp) fclose(fp);
    }
};

// slot s of every block, copied to the host
amr_status slot_to_host(amr_forest *f, int s, std::vector<char> &out, cudaStream_t st) {
    out.resize(size_t(nblocks(f)) * f->block_bytes);
    if (!out.empty()) CU(cudaMemcpyAsync(out.data(), slot_ptr(f, s), out.size(), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return AMR_OK;
}

}  // namespace

extern "C" {

amr_status amr_get_config(const amr_forest *f, int inst, amr_config *out) {
    if (!f || !out || inst < 0 || inst >= n_inst(f)) return AMR_EINVAL;
    *out = f->icfg[size_t(inst)];
    return AMR_OK;
}

amr_status amr_save(const amr_forest *fc, const char *path, amr_stream stream) {
    if (!fc || !path) return AMR_EINVAL;
    amr_forest *f = const_cast<amr_forest *>(fc);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ni = n_inst(f);
    std::vector<double> dts(size_t(ni), 0.0);
    std::vector<char> state;
    if (!f->cfg.host_only) {
        std::vector<DevScalars> sc(static_cast<size_t>(ni));
        CU(cudaMemcpyAsync(sc.data(), f->sc.p, sizeof(DevScalars) * size_t(ni), cudaMemcpyDeviceToHost, st));
        amr_status r = slot_to_host(f, 0, state, st);
        if (r != AMR_OK) return r;
        for (int i = 0; i < ni; ++i) dts[size_t(i)] = sc[size_t(i)].dt;
    }
    CFile out;
    out.fp = fopen(path, "wb");
    if (!out.fp) return fail(f, AMR_ESTATE, "cannot open %s for writing", path);
    CkptHead h{};
    memcpy(h.magic, kCkptMagic, 8);
    h.version = kCkptVersion;
    h.n_inst = uint32_t(ni);
    const amr_config &c0 = f->cfg;
    h.precision = c0.precision;
    h.ndim = c0.ndim;
    h.block_n = c0.block_n;
    h.n_ghost = c0.n_ghost;
    h.n_var = c0.n_var;
    h.n_states = c0.n_states;
    h.host_only = c0.host_only;
    h.limiter = c0.limiter;
    h.flux = c0.flux;
    h.diagonal_ghosts = c0.diagonal_ghosts;
    h.gamma = c0.gamma;
    for (int d = 0; d < 3; ++d) h.gravity[d] = c0.gravity[d];
    h.physics = c0.physics;
    for (int d = 0; d < 3; ++d) h.velocity[d] = c0.velocity[d];
    h.n_blocks = nblocks(f);
    bool ok = fwrite(&h, sizeof h, 1, out.fp) == 1;
    for (int i = 0; i < ni && ok; ++i) {
        const amr_config &c = f->icfg[size_t(i)];
        CkptInst r{};
        for (int d = 0; d < 3; ++d) {
            r.ntrees[d] = c.ntrees[d];
            r.periodic[d] = c.periodic[d];
            r.lo[d] = c.lo[d];
            r.len[d] = c.len[d];
        }
        r.max_level = c.max_level;
        r.max_blocks = c.max_blocks;
        for (int q = 0; q < 6; ++q) {
            r.bc[q] = c.bc[q];
            for (int v = 0; v < 8; ++v) r.bc_val[q][v] = c.bc_val[q][v];
        }
        r.cfl = c.cfl;
        r.dt = dts[size_t(i)];
        const std::vector<Leaf> &L = f->inst[size_t(i)].leaves;
        r.n_leaves = int64_t(L.size());
        ok = fwrite(&r, sizeof r, 1, out.fp) == 1;
        std::vector<CkptLeaf> lv(L.size());
        for (size_t b = 0; b < L.size(); ++b) {
            lv[b].lev = L[b].lev;
            for (int d = 0; d < 3; ++d) lv[b].g[d] = L[b].g[d];
        }
        if (ok && !lv.empty()) ok = fwrite(lv.data(), sizeof(CkptLeaf), lv.size(), out.fp) == lv.size();
    }
    if (ok && !state.empty()) ok = fwrite(state.data(), 1, state.size(), out.fp) == state.size();
    if (!ok || fflush(out.fp) != 0) return fail(f, AMR_ESTATE, "short write to %s", path);
    return AMR_OK;
}

amr_status amr_load(const char *path, const amr_config *opts, amr_forest **out, amr_stream stream) {
    if (!path || !out) return AMR_EINVAL;
    *out = nullptr;
    CFile in;
    in.fp = fopen(path, "rb");
    if (!in.fp) return AMR_ESTATE;
    CkptHead h{};
    if (fread(&h, sizeof h, 1, in.fp) != 1 || memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != kCkptVersion ||
        h.n_inst < 1 || h.n_inst > (1u << 20) || h.n_blocks < 0)
        return AMR_ESTATE;
    const int ni = int(h.n_inst);
    std::vector<amr_config> cfgs(static_cast<size_t>(ni));
    std::vector<double> dts(static_cast<size_t>(ni));
    std::vector<std::vector<Leaf>> leaves(static_cast<size_t>(ni));
    const int host_only = opts ? opts->host_only : 0;
    if (!host_only && h.host_only) return AMR_ESTATE;   // a mesh-only checkpoint has no state
    int64_t total = 0;
    for (int i = 0; i < ni; ++i) {
        CkptInst r{};
        if (fread(&r, sizeof r, 1, in.fp) != 1 || r.n_leaves < 1 || r.n_leaves > (int64_t(1) << 31)) return AMR_ESTATE;
        amr_config &c = cfgs[size_t(i)];
        c = amr_config{};
        c.ndim = h.ndim;
        c.block_n = h.block_n;
        c.n_ghost = h.n_ghost;
        c.n_var = h.n_var;
        c.precision = h.precision;
        c.gamma = h.gamma;
        c.limiter = h.limiter;
        c.flux = h.flux;
        c.diagonal_ghosts = h.diagonal_ghosts;
        c.physics = h.physics;
        for (int d = 0; d < 3; ++d) {
            c.velocity[d] = h.velocity[d];
            c.gravity[d] = h.gravity[d];
            c.ntrees[d] = r.ntrees[d];
            c.periodic[d] = r.periodic[d];
            c.lo[d] = r.lo[d];
            c.len[d] = r.len[d];
        }
        c.max_level = r.max_level;
        c.max_blocks = r.max_blocks;
        c.cfl = r.cfl;
        for (int q = 0; q < 6; ++q) {
            c.bc[q] = r.bc[q];
            for (int v = 0; v < 8; ++v) c.bc_val[q][v] = r.bc_val[q][v];
        }
        c.n_states = opts ? opts->n_states : h.n_states;
        c.host_only = host_only;
        if (opts) {
            c.dev_alloc = opts->dev_alloc;
            c.dev_free = opts->dev_free;
            c.alloc_ctx = opts->alloc_ctx;
        }
        dts[size_t(i)] = r.dt;
        std::vector<CkptLeaf> lv(size_t(r.n_leaves));
        if (fread(lv.data(), sizeof(CkptLeaf), lv.size(), in.fp) != lv.size()) return AMR_ESTATE;
        std::vector<Leaf> &L = leaves[size_t(i)];
        L.resize(lv.size());
        for (size_t b = 0; b < lv.size(); ++b) {
            if (lv[b].lev < 0 || lv[b].lev > c.max_level) return AMR_ESTATE;
            L[b].lev = lv[b].lev;
            for (int d = 0; d < 3; ++d) {
                const int64_t E = int64_t(d < c.ndim ? c.ntrees[d] : 1) << (d < c.ndim ? lv[b].lev : 0);
                const int64_t x = d < c.ndim ? lv[b].g[d] : 0;
                if (x < 0 || x >= E) return AMR_ESTATE;
                L[b].g[d] = x;
            }
        }
        if (int64_t(L.size()) > c.max_blocks) return AMR_ECAPACITY;
        total += int64_t(L.size());
    }
    if (total != h.n_blocks) return AMR_ESTATE;
    std::vector<int> levels(size_t(ni), 0);
    amr_forest *f = nullptr;
    amr_status r = amr_create_batch(cfgs.data(), levels.data(), ni, &f);
    if (r != AMR_OK) return r;
    for (int i = 0; i < ni; ++i) {
        std::vector<Leaf> saved = leaves[size_t(i)];
        f->inst[size_t(i)].assign(std::move(leaves[size_t(i)]));
        const std::vector<Leaf> &now = f->inst[size_t(i)].leaves;
        bool same = now.size() == saved.size();
        for (size_t b = 0; same && b < now.size(); ++b)
            same = now[b].lev == saved[b].lev && now[b].g[0] == saved[b].g[0] && now[b].g[1] == saved[b].g[1] &&
                   now[b].g[2] == saved[b].g[2];
        if (!same) {   // not a leaf list this library wrote (block order)
            amr_destroy_forest(f);
            return AMR_ESTATE;
        }
    }
    set_offsets(f);
    ++f->revision;
    if ((r = upload_pattern(f)) != AMR_OK) {
        amr_destroy_forest(f);
        return r;
    }
    if (!host_only) {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        std::vector<char> state(size_t(total) * f->block_bytes);
        std::vector<DevScalars> sc(static_cast<size_t>(ni));
        bool ok = h.host_only == 0 && (state.empty() || fread(state.data(), 1, state.size(), in.fp) == state.size());
        if (ok && !state.empty()) ok = cudaMemcpyAsync(slot_ptr(f, 0), state.data(), state.size(), cudaMemcpyHostToDevice, st) == cudaSuccess;
        if (ok) ok = cudaMemcpyAsync(sc.data(), f->sc.p, sizeof(DevScalars) * size_t(ni), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                     cudaStreamSynchronize(st) == cudaSuccess;
        for (int i = 0; ok && i < ni; ++i) sc[size_t(i)].dt = dts[size_t(i)];
        if (ok) ok = cudaMemcpyAsync(f->sc.p, sc.data(), sizeof(DevScalars) * size_t(ni), cudaMemcpyHostToDevice, st) == cudaSuccess &&
                     cudaStreamSynchronize(st) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            amr_destroy_forest(f);
            return AMR_ESTATE;
        }
    }
    *out = f;
    return AMR_OK;
}

amr_status amr_write_xdmf(const amr_forest *fc, int s, const char *base, amr_stream stream) {
    if (!fc || !base || !valid_slot(fc, s)) return AMR_EINVAL;
    amr_forest *f = const_cast<amr_forest *>(fc);
    NEED_DEVICE(f);
    std::vector<char> state;
    amr_status r = slot_to_host(f, s, state, static_cast<cudaStream_t>(stream));
    if (r != AMR_OK) return r;
    const int D = f->cfg.ndim, N = f->cfg.block_n, V = f->cfg.n_var;
    const int64_t S = f->geom.S, ng = f->cfg.n_ghost;
    const int64_t nint = D == 3 ? int64_t(N) * N * N : int64_t(N) * N;
    const size_t es = size_t(f->esize);
    const std::string bin = std::string(base) + ".bin", xmf = std::string(base) + ".xmf";
    std::string binname = bin;
    const size_t slash = binname.find_last_of('/');
    if (slash != std::string::npos) binname = binname.substr(slash + 1);
    {
        CFile out;
        out.fp = fopen(bin.c_str(), "wb");
        if (!out.fp) return fail(f, AMR_ESTATE, "cannot open %s", bin.c_str());
        std::vector<char> buf(size_t(nint) * es);
        for (int64_t b = 0; b < nblocks(f); ++b)
            for (int v = 0; v < V; ++v) {
                const char *blk = state.data() + size_t(b) * f->block_bytes + size_t(v) * size_t(f->geom.ncell) * es;
                size_t o = 0;
                for (int k = 0; k < (D == 3 ? N : 1); ++k)
                    for (int j = 0; j < N; ++j) {
                        const int64_t row = ((D == 3 ? k + ng : 0) * S + (j + ng)) * S + ng;
                        memcpy(buf.data() + o, blk + size_t(row) * es, size_t(N) * es);
                        o += size_t(N) * es;
                    }
                if (fwrite(buf.data(), 1, buf.size(), out.fp) != buf.size()) return fail(f, AMR_ESTATE, "short write to %s", bin.c_str());
            }
    }
    CFile out;
    out.fp = fopen(xmf.c_str(), "w");
    if (!out.fp) return fail(f, AMR_ESTATE, "cannot open %s", xmf.c_str());
    static const char *names3[5] = {"rho", "mx", "my", "mz", "E"};
    static const char *names2[4] = {"rho", "mx", "my", "E"};
    static const char *names1[1] = {"rho"};
    const char **names = f->cfg.physics == AMR_PHYS_ADVECTION ? names1 : (D == 3 ? names3 : names2);
    // co-rectilinear grids: dimensions (node counts), origin and spacing are
    // all listed slowest dimension first (z, y, x)
    fprintf(out.fp, "<?xml version=\"1.0\" ?>\n<Xdmf Version=\"2.0\">\n <Domain>\n");
    int64_t b = 0;
    for (int i = 0; i < n_inst(f); ++i) {
        const amr_config &c = f->icfg[size_t(i)];
        fprintf(out.fp, "  <Grid Name=\"instance%d\" GridType=\"Collection\" CollectionType=\"Spatial\">\n", i);
        for (const Leaf &l : f->inst[size_t(i)].leaves) {
            double org[3], dx[3];
            for (int d = 0; d < D; ++d) {
                dx[d] = c.len[d] / double(c.ntrees[d]) / (double(N) * double(int64_t(1) << l.lev));
                org[d] = c.lo[d] + double(l.g[d]) * double(N) * dx[d];
            }
            fprintf(out.fp, "   <Grid Name=\"b%lld\" GridType=\"Uniform\">\n", (long long)b);
            if (D == 3) {
                fprintf(out.fp, "    <Topology TopologyType=\"3DCoRectMesh\" Dimensions=\"%d %d %d\"/>\n", N + 1, N + 1, N + 1);
                fprintf(out.fp, "    <Geometry GeometryType=\"ORIGIN_DXDYDZ\">\n");
                fprintf(out.fp, "     <DataItem Dimensions=\"3\" Format=\"XML\">%.17g %.17g %.17g</DataItem>\n", org[2], org[1], org[0]);
                fprintf(out.fp, "     <DataItem Dimensions=\"3\" Format=\"XML\">%.17g %.17g %.17g</DataItem>\n", dx[2], dx[1], dx[0]);
            } else {
                fprintf(out.fp, "    <Topology TopologyType=\"2DCoRectMesh\" Dimensions=\"%d %d\"/>\n", N + 1, N + 1);
                fprintf(out.fp, "    <Geometry GeometryType=\"ORIGIN_DXDY\">\n");
                fprintf(out.fp, "     <DataItem Dimensions=\"2\" Format=\"XML\">%.17g %.17g</DataItem>\n", org[1], org[0]);
                fprintf(out.fp, "     <DataItem Dimensions=\"2\" Format=\"XML\">%.17g %.17g</DataItem>\n", dx[1], dx[0]);
            }
            fprintf(out.fp, "    </Geometry>\n");
            for (int v = 0; v < V; ++v) {
                const long long seek = (long long)((b * V + v) * nint) * (long long)es;
                fprintf(out.fp, "    <Attribute Name=\"%s\" AttributeType=\"Scalar\" Center=\"Cell\">\n", names[v]);
                if (D == 3)
                    fprintf(out.fp, "     <DataItem Dimensions=\"%d %d %d\"", N, N, N);
                else
                    fprintf(out.fp, "     <DataItem Dimensions=\"%d %d\"", N, N);
                fprintf(out.fp, " NumberType=\"Float\" Precision=\"%d\" Format=\"Binary\" Endian=\"Little\" Seek=\"%lld\">%s</DataItem>\n",
                        int(es), seek, binname.c_str());
                fprintf(out.fp, "    </Attribute>\n");
            }
            fprintf(out.fp, "   </Grid>\n");
            ++b;
        }
        fprintf(out.fp, "  </Grid>\n");
    }
    fprintf(out.fp, " </Domain>\n</Xdmf>\n");
    if (ferror(out.fp) || fflush(out.fp) != 0) return fail(f, AMR_ESTATE, "short write to %s", xmf.c_str());
    return AMR_OK;
}

}  // extern "C"

extern "C" {

const char *amr_last_error(const amr_forest *f) { return f ? f->err.c_str() : "null forest"; }

amr_status amr_launch_count(const amr_forest *f, int64_t *n) {
    if (!f || !n) return AMR_EINVAL;
    *n = f->launches;
    return AMR_OK;
}

amr_status amr_trace(amr_forest *f, int on) {
    if (!f) return AMR_EINVAL;
    f->tracing = on != 0;
    return AMR_OK;
}

amr_status amr_trace_read(amr_forest *f, double *ms, int64_t *count, int reset) {
    if (!f) return AMR_EINVAL;
    const bool ok = trace_drain(f) && !f->trace_lost;
    if (reset) f->trace_lost = false;
    for (int p = 0; p < AMR_N_PHASES; ++p) {
        if (ms) ms[p] = f->trace_ms[p];
        if (count) count[p] = f->trace_n[p];
        if (reset) {
            f->trace_ms[p] = 0.0;
            f->trace_n[p] = 0;
        }
    }
    return ok ? AMR_OK : fail(f, AMR_ECUDA, "trace: a recorded phase could not be timed (dropped)");
}

}  // extern "C"
