// Definitions of the ghost and stage kernel launchers declared in
// api_internal.cuh; the inst_*.cu units instantiate them.
#pragma once
#include <atomic>
#include <type_traits>

#include "api_internal.cuh"
#include "ghost.cuh"
#include "stage.cuh"
#include "stage_pair.cuh"
#include "stage_pair2d.cuh"
#include "stage_adv.cuh"
#include "stage_weno.cuh"

namespace amrb {

// The dynamic shared-memory limit of a kernel is a per-device setting: it is
// raised once per (kernel, device) -- `done` holds one bit per device id.
template <class K>
cudaError_t smem_attr_once(K kern, size_t smem, std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
    return e;
}

template <class real, int D>
amr_status launch_ghosts(amr_forest *f, int s, cudaStream_t st, bool gather) {
    GhostArgs<real> a{};
    a.u = static_cast<real *>(slot_ptr(f, s));
    a.bcdata = static_cast<const real *>(f->bcdata.p);
    a.bc_type = static_cast<const int32_t *>(f->bctype.p);
    a.bc_val = static_cast<const real *>(f->bcval.p);
    a.info = static_cast<const BlockInfo *>(f->info.p);
    // rounds 1 and 2, then the edge and the corner regions outside the domain
    const int n3 = int(f->pat.round3.size()), n3e = f->pat.n_round3_edges;
    for (int round = 0; round < 4; ++round) {
        const Entry *list;
        int n;
        if (round < 2) {
            const auto &lst = round == 0 ? (gather ? f->pat.round1_gather : f->pat.round1) : f->pat.round2;
            list = static_cast<const Entry *>(round == 0 ? (gather ? f->r1g.p : f->r1.p) : f->r2.p);
            n = int(lst.size());
        } else {
            list = static_cast<const Entry *>(f->r3.p) + (round == 3 ? n3e : 0);
            n = round == 2 ? n3e : n3 - n3e;
        }
        if (n == 0) continue;
        a.list = list;
        a.n = n;
        const int N = f->cfg.block_n, NG = f->cfg.n_ghost;
        // warps per strip: about 512 values of a full face strip each
        const int64_t face_vals = int64_t(D == 3 ? N * N : N) * NG * f->cfg.n_var;
        a.parts = int(std::max<int64_t>(1, std::min<int64_t>(32, face_vals / 512)));
        const int64_t grid = (int64_t(a.n) * a.parts + 7) / 8;
        // the edge and corner launches after round 2 are timed as round 2
        TraceSpan span(f, round == 0 ? AMR_PHASE_GHOST_R1 : AMR_PHASE_GHOST_R2, st);
        bool launched = false;
#define AMR_GHOST_CASE(n_, g_)                                                   \
    if (!launched && N == n_ && NG == g_) {                                     \
        k_ghost<real, D, n_, g_><<<unsigned(grid), 256, 0, st>>>(a, f->geom);             \
        launched = true;                                                        \
    }
        AMR_GHOST_CASE(8, 1) AMR_GHOST_CASE(8, 2) AMR_GHOST_CASE(8, 3) AMR_GHOST_CASE(8, 4)
        AMR_GHOST_CASE(16, 1) AMR_GHOST_CASE(16, 2) AMR_GHOST_CASE(16, 3) AMR_GHOST_CASE(16, 4)
        AMR_GHOST_CASE(32, 1) AMR_GHOST_CASE(32, 2) AMR_GHOST_CASE(32, 3) AMR_GHOST_CASE(32, 4)
#undef AMR_GHOST_CASE
        if (!launched) return fail(f, AMR_EINVAL, "no ghost kernel for block_n %d, n_ghost %d", N, NG);
        ++f->launches;
    }
    CU(cudaGetLastError());
    return AMR_OK;
}

template <class real, int D, int N, int NG, bool GEN, int PH>
amr_status launch_stage_t(amr_forest *f, const StageArgs<real> &a, cudaStream_t st) {
    constexpr int T = N < 16 ? N : 16;
    using Sh = StageShape<real, D, N, NG, T, PH>;
    constexpr auto kern = k_stage<real, D, N, NG, T, GEN, PH>;
    static std::atomic<unsigned long long> attr_done{0};
    const size_t smem = Sh::smem_bytes();
    CU(smem_attr_once(kern, smem, attr_done));
    const int64_t items = nblocks(f) * Sh::TILES;
    if (items > 0) {
        StageArgs<real> b = a;
        b.n_items = int(items);
        int occ = 1;
        if (f->persistent) CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, Sh::NT, smem));
        const int64_t grid = stage_grid(f, items, occ);
        kern<<<unsigned(grid), Sh::NT, smem, st>>>(b, f->geom);
        ++f->launches;
    }
    CU(cudaGetLastError());
    return AMR_OK;
}

// FP32, two ghost layers: the packed cell-pair kernels (3D plane march, 2D
// single plane), specialised for one and two previous states (the two stages
// of Heun's method), for the slope limiter (minmod, MC, van Leer), the flux
// (Rusanov, HLL) and the staging tile (16, or 8 when the autotuner picks it
// for blocks above 8 cells a side)
// (3D: FIX = the mesh has refinement faces; the 2D kernel has one form)
template <int D, int N, int TT, int NPREV, int LIM, int FLX, bool FIX>
struct PairKernel;
template <int N, int TT, int NPREV, int LIM, int FLX, bool FIX>
struct PairKernel<3, N, TT, NPREV, LIM, FLX, FIX> {
    using Sh = PairShape<N, TT>;
    static constexpr auto fn = k_stage_pair<N, TT, NPREV, LIM, FLX, FIX>;
};
template <int N, int TT, int NPREV, int LIM, int FLX, bool FIX>
struct PairKernel<2, N, TT, NPREV, LIM, FLX, FIX> {
    using Sh = PairShape2D<N, TT>;
    static constexpr auto fn = k_stage_pair2d<N, TT, NPREV, LIM, FLX>;
};

// the mesh has refinement faces: flux stores and flux fixing
inline bool has_refinement_faces(const amr_forest *f) { return f->pat.n_slots > 0 || f->pat.fix_start.size() > 1; }

template <int D, int N, int TT, int NPREV, int LIM, int FLX, bool FIX>
amr_status launch_stage_pair_f(amr_forest *f, const StageArgs<float> &a, cudaStream_t st) {
    using K = PairKernel<D, N, TT, NPREV, LIM, FLX, FIX>;
    using Sh = typename K::Sh;
    static std::atomic<unsigned long long> attr_done{0};
    const size_t smem = Sh::smem_bytes(NPREV);
    CU(smem_attr_once(K::fn, smem, attr_done));
    const int64_t items = nblocks(f) * Sh::TILES;
    if (items > 0) {
        StageArgs<float> b = a;
        b.n_items = int(items);
        int occ = 1;
        if (f->persistent) CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, K::fn, Sh::NT, smem));
        const int64_t grid = stage_grid(f, items, occ);
        K::fn<<<unsigned(grid), Sh::NT, smem, st>>>(b, f->geom);
        ++f->launches;
    }
    CU(cudaGetLastError());
    return AMR_OK;
}

template <int D, int N, int TT, int NPREV, int LIM, int FLX>
amr_status launch_stage_pair_n(amr_forest *f, const StageArgs<float> &a, cudaStream_t st) {
    if constexpr (D == 2) {
        return launch_stage_pair_f<D, N, TT, NPREV, LIM, FLX, true>(f, a, st);
    } else {
        if (has_refinement_faces(f)) return launch_stage_pair_f<D, N, TT, NPREV, LIM, FLX, true>(f, a, st);
        return launch_stage_pair_f<D, N, TT, NPREV, LIM, FLX, false>(f, a, st);
    }
}

template <int D, int N, int TT, int LIM, int FLX>
amr_status launch_stage_pair_l(amr_forest *f, const StageArgs<float> &a, cudaStream_t st) {
    if (a.nprev == 1) return launch_stage_pair_n<D, N, TT, 1, LIM, FLX>(f, a, st);
    if (a.nprev == 2) return launch_stage_pair_n<D, N, TT, 2, LIM, FLX>(f, a, st);
    return launch_stage_pair_n<D, N, TT, -1, LIM, FLX>(f, a, st);
}

template <int D, int N, int TT, int FLX>
amr_status launch_stage_pair_t(amr_forest *f, const StageArgs<float> &a, cudaStream_t st) {
    if (a.limiter == AMR_LIM_MC) return launch_stage_pair_l<D, N, TT, 1, FLX>(f, a, st);
    if (a.limiter == AMR_LIM_VANLEER) return launch_stage_pair_l<D, N, TT, 2, FLX>(f, a, st);
    return launch_stage_pair_l<D, N, TT, 0, FLX>(f, a, st);
}

// FLX 0: Rusanov, 1: HLL (separate build units)
template <int D, int N, int FLX>
amr_status launch_stage_pair(amr_forest *f, const StageArgs<float> &a, cudaStream_t st) {
    if constexpr (N > 8) {
        if (f->pair_tile == 8) return launch_stage_pair_t<D, N, 8, FLX>(f, a, st);
    }
    return launch_stage_pair_t<D, N, (N < 16 ? N : 16), FLX>(f, a, st);
}

// FP32 scalar advection with a MUSCL slope limiter: one CTA per block (the
// block and its face halo in shared memory)
template <int D, int N, int LIM, int NPREV>
amr_status launch_adv_pair_n(amr_forest *f, const StageArgs<float> &a, cudaStream_t st) {
    using Sh = AdvShape<D, N>;
    constexpr auto kern = k_adv_pair<D, N, LIM, NPREV>;
    static std::atomic<unsigned long long> attr_done{0};
    const size_t smem = Sh::smem_bytes();
    CU(smem_attr_once(kern, smem, attr_done));
    const int64_t items = nblocks(f);
    if (items > 0) {
        StageArgs<float> b = a;
        b.n_items = int(items);
        int occ = 1;
        if (f->persistent) CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, Sh::NT, smem));
        const int64_t grid = stage_grid(f, items, occ);
        kern<<<unsigned(grid), Sh::NT, smem, st>>>(b, f->geom);
        ++f->launches;
    }
    CU(cudaGetLastError());
    return AMR_OK;
}

template <int D, int N, int LIM>
amr_status launch_adv_pair_l(amr_forest *f, const StageArgs<float> &a, cudaStream_t st) {
    if (a.nprev == 1) return launch_adv_pair_n<D, N, LIM, 1>(f, a, st);
    if (a.nprev == 2) return launch_adv_pair_n<D, N, LIM, 2>(f, a, st);
    return launch_adv_pair_n<D, N, LIM, -1>(f, a, st);
}

template <int D, int N>
amr_status launch_adv_pair(amr_forest *f, const StageArgs<float> &a, cudaStream_t st) {
    if (a.limiter == AMR_LIM_MC) return launch_adv_pair_l<D, N, 1>(f, a, st);
    if (a.limiter == AMR_LIM_VANLEER) return launch_adv_pair_l<D, N, 2>(f, a, st);
    return launch_adv_pair_l<D, N, 0>(f, a, st);
}

// WENO5 stage: face fluxes, then the update (two launches); flux is a
// scratch buffer of n_blocks x D x V x (N+1) N^(D-1) elements
template <int N, int PH>
cudaError_t launch_weno_fused(amr_forest *f, const StageArgs<float> &a, const PhysCtx<float> &pc, cudaStream_t st) {
    using W = WenoFused<N, PH>;
    static std::atomic<unsigned long long> attr_done{0};
    cudaError_t e = smem_attr_once(k_weno_fused<N, PH>, W::smem_bytes(), attr_done);
    if (e != cudaSuccess) return e;
    int occ = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_weno_fused<N, PH>, W::NT, W::smem_bytes());
    if (e != cudaSuccess) return e;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.n_items, int64_t(f->n_sms) * std::max(occ, 1)));
    k_weno_fused<N, PH><<<unsigned(grid), W::NT, W::smem_bytes(), st>>>(a, f->geom, pc);
    return cudaGetLastError();
}

template <class real, int D, int PH>
amr_status launch_weno(amr_forest *f, const StageArgs<real> &a, real *flux, cudaStream_t st) {
    const int64_t nb = nblocks(f);
    if constexpr (std::is_same<real, float>::value && D == 3) {
        if (weno_fused_applies(f)) {
            const PhysCtx<float> pc{a.gamma, 1.f / (a.gamma - 1.f), {a.vel[0], a.vel[1], a.vel[2]}};
            StageArgs<float> b = a;
            b.n_items = int(nb);
            if (nb > 0) {
                const cudaError_t e = f->cfg.block_n == 16 ? launch_weno_fused<16, PH>(f, b, pc, st)
                                                           : launch_weno_fused<8, PH>(f, b, pc, st);
                CU(e);
                f->launches += 1;
            }
            CU(cudaGetLastError());
            return AMR_OK;
        }
    }
    if (nb > 0) {
        const int N = f->cfg.block_n;
        const int npen = D * (D == 3 ? N * N : N);   // pencils of faces (one thread each)
        const int ncint = D == 3 ? N * N * N : N * N;
        const PhysCtx<real> pc{a.gamma, real(1) / (a.gamma - real(1)), {a.vel[0], a.vel[1], a.vel[2]}};
        // one-dimensional grids: a block's chunks are consecutive CTAs
        k_weno_flux<real, D, PH><<<unsigned(nb * ((npen + 255) / 256)), 256, 0, st>>>(a.deriv, flux, a.info, a.bflux,
                                                                                   f->geom, pc, a.flux, a.sc);
        k_weno_update<real, D, PH><<<unsigned(nb * ((ncint + 255) / 256)), 256, 0, st>>>(a, flux, f->geom);
        f->launches += 2;
    }
    CU(cudaGetLastError());
    return AMR_OK;
}

}  // namespace amrb

#define AMR_INST_STAGE_PH(real, D, GEN, PH)                                                                 \
    template amr_status launch_stage_t<real, D, 8, 2, GEN, PH>(amr_forest *, const StageArgs<real> &, cudaStream_t);  \
    template amr_status launch_stage_t<real, D, 16, 2, GEN, PH>(amr_forest *, const StageArgs<real> &, cudaStream_t); \
    template amr_status launch_stage_t<real, D, 32, 2, GEN, PH>(amr_forest *, const StageArgs<real> &, cudaStream_t); \
    template amr_status launch_stage_t<real, D, 8, 3, GEN, PH>(amr_forest *, const StageArgs<real> &, cudaStream_t);  \
    template amr_status launch_stage_t<real, D, 16, 3, GEN, PH>(amr_forest *, const StageArgs<real> &, cudaStream_t); \
    template amr_status launch_stage_t<real, D, 32, 3, GEN, PH>(amr_forest *, const StageArgs<real> &, cudaStream_t);
#define AMR_INST_STAGE(real, D, GEN) AMR_INST_STAGE_PH(real, D, GEN, 0)
