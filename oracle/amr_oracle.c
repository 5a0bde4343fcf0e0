/*
 * amr_oracle.c -- plain, slow, FP64 CPU oracle of the block-AMR hot path of
 * "foap4: adaptive mesh refinement with OpenACC, MPI, and p4est".
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library; the two meet only in the seeded
 * input generators (package `synth`) and in the comparisons the tests make.
 *
 * Everything is written for reading, not for speed: meshes are flat leaf lists
 * plus a hash of (level, coordinates); ghost cells are filled one cell at a
 * time by locating the leaf that holds the cell; fluxes are recomputed per
 * face.  Compiled with -O2 -ffp-contract=off so that every product and sum is
 * rounded exactly as written.
 *
 * Readings of points the paper leaves open (all fixed here, the CUDA side
 * follows the same readings):
 *   - leaf order: trees row-major (x fastest), Morton order inside a tree
 *     with x the lowest bit (Sec. 2.2: the n-th quadrant is the n-th block);
 *   - restriction sums x-pairs, then y-pairs, then z-pairs, then scales by
 *     2^-d (Sec. 2.2 "average of the fine values");
 *   - prolongation adds the per-dimension corrections left to right before
 *     adding them to the coarse value (Sec. 2.2, Eq. 1 with theta = 1);
 *   - Dirichlet ghost = 2 u_b - u_mirror, Neumann ghost = u_mirror +
 *     (2k-1) dx u'_b for the k-th layer (Sec. 2.4, formulas not printed);
 *   - Rusanov flux with the Einfeldt speed |u_roe| + d_roe (Sec. 3.2-3.5);
 *   - dt = CFL / max over leaf cells of sum_d (|v_d| + c) / dx_d (Sec. 3.2);
 *   - flux fixing is applied after every Runge-Kutta stage with that stage's
 *     time step (Sec. 2.7);
 *   - scalar advection (Sec. 3.4) uses the same flux schemes with the wave
 *     speeds min(v_n, 0), max(v_n, 0); its HLL flux is 0 where v_n = 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Parameters and mesh                                                       */
/* ------------------------------------------------------------------------ */

/* Mirrors the problem statement of Sec. 2.2-2.4: a brick of ntrees[0] x
 * ntrees[1] (x ntrees[2]) trees (Sec. 2.2), blocks of N^d cells plus ng ghost
 * layers (Sec. 2.3, Eq. 3), boundary type per face direction in the order
 * -x,+x,-y,+y,-z,+z (Sec. 2.4). */
typedef struct {
    int ndim, N, ng, nvar;
    int ntrees[3];
    int periodic[3];
    double lo[3], len[3];
    int max_level;
    double gamma, cfl;
    int bc_type[6];        /* 0 periodic/none, 1 Dirichlet, 2 Neumann, 3 Dirichlet from bc_data */
    double bc_val[6][8];
    int limiter;           /* face reconstruction (Sec. 3.2 list): 0 minmod, 1 MC, 2 van Leer
                              (MUSCL slopes), 3 WENO5 (needs ng >= 3), 4 Koren,
                              5 WENO3, 6 first-order upwind */
    int flux;              /* 0 Rusanov, 1 HLL (Sec. 3.2 list), both with Einfeldt speeds */
    double gravity[3];     /* g of the source term S = (0, rho g, rho g.u) (Sec. 4.2) */
    int diagonal;          /* 1: also fill edge and corner ghost cells (copy from a
                              same-level leaf, restriction from finer, prolongation
                              from coarser ones); the paper fills face ghosts only */
    int physics;           /* 0 Euler gas dynamics (Sec. 3.5), 1 scalar advection
                              (Sec. 3.4, Eq. 13; nvar = 1) */
    double velocity[3];    /* the uniform advection velocity v of Eq. 13 */
} orc_params;

enum { BC_NONE = 0, BC_DIRICHLET = 1, BC_NEUMANN = 2, BC_DATA = 3 };
enum { K_SRL = 0, K_F2C = 1, K_BC = 2, K_C2F = 3, K_DIAG = 4, K_DIAG_F2C = 5, K_DIAG_C2F = 6, K_DIAG_BC = 7 };

/* a diagonal (edge or corner) direction (dx, dy, dz), two or three of them
 * nonzero, as the code (dx+1) + 3 (dy+1) + 9 (dz+1) */
static int diag_code(const int dir[3]) { return (dir[0] + 1) + 3 * (dir[1] + 1) + 9 * (dir[2] + 1); }

#define ORDER_DEPTH 20     /* Morton depth used to order leaves of any level */

typedef struct {
    orc_params p;
    int n;                 /* number of leaves = number of blocks */
    int *lev;              /* [n] refinement level */
    int64_t *g;            /* [n][3] block coordinates at the leaf's own level, over the whole brick */
    int64_t hcap;
    uint64_t *hk;          /* hash keys, ~0 = empty */
    int *hv;               /* leaf index */
} orc_mesh;

static uint64_t key_of(int lev, const int64_t g[3])
{
    return ((uint64_t)lev << 57) | ((uint64_t)g[2] << 38) | ((uint64_t)g[1] << 19) | (uint64_t)g[0];
}

static uint64_t hash64(uint64_t x)
{
    x ^= x >> 33; x *= 0xff51afd7ed558ccdULL; x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL; x ^= x >> 33;
    return x;
}

static void hash_build(orc_mesh *m)
{
    m->hcap = 16;
    while (m->hcap < 4 * (int64_t)m->n) m->hcap *= 2;
    m->hk = (uint64_t *)malloc(sizeof(uint64_t) * m->hcap);
    m->hv = (int *)malloc(sizeof(int) * m->hcap);
    for (int64_t i = 0; i < m->hcap; i++) m->hk[i] = ~0ULL;
    for (int b = 0; b < m->n; b++) {
        uint64_t k = key_of(m->lev[b], &m->g[3 * b]);
        int64_t s = (int64_t)(hash64(k) & (uint64_t)(m->hcap - 1));
        while (m->hk[s] != ~0ULL) s = (s + 1) & (m->hcap - 1);
        m->hk[s] = k;
        m->hv[s] = b;
    }
}

/* Leaf index of the block (lev, g), or -1 if that block is not a leaf. */
static int find_leaf(const orc_mesh *m, int lev, const int64_t g[3])
{
    uint64_t k = key_of(lev, g);
    int64_t s = (int64_t)(hash64(k) & (uint64_t)(m->hcap - 1));
    while (m->hk[s] != ~0ULL) {
        if (m->hk[s] == k) return m->hv[s];
        s = (s + 1) & (m->hcap - 1);
    }
    return -1;
}

static int64_t blocks_at(const orc_params *p, int d, int lev)
{
    return (int64_t)p->ntrees[d] << lev;
}

/* ---- leaf order (Sec. 2.2) ---- */
typedef struct { int lev; int64_t g[3]; int64_t tree; uint64_t morton; } leaf_t;

static void order_key(const orc_params *p, leaf_t *L)
{
    int64_t t[3] = {0, 0, 0}, loc[3] = {0, 0, 0};
    for (int d = 0; d < p->ndim; d++) {
        t[d] = L->g[d] >> L->lev;
        loc[d] = (L->g[d] - (t[d] << L->lev)) << (ORDER_DEPTH - L->lev);
    }
    L->tree = t[0] + (int64_t)p->ntrees[0] * (t[1] + (int64_t)p->ntrees[1] * t[2]);
    uint64_t mk = 0;
    for (int b = 0; b < ORDER_DEPTH; b++)
        for (int d = 0; d < p->ndim; d++)
            mk |= (uint64_t)((loc[d] >> b) & 1) << (p->ndim * b + d);
    L->morton = mk;
}

static int cmp_leaf(const void *a, const void *b)
{
    const leaf_t *x = (const leaf_t *)a, *y = (const leaf_t *)b;
    if (x->tree != y->tree) return x->tree < y->tree ? -1 : 1;
    if (x->morton != y->morton) return x->morton < y->morton ? -1 : 1;
    return 0;
}

static orc_mesh *mesh_from_leaves(const orc_params *p, leaf_t *L, int n)
{
    for (int i = 0; i < n; i++) order_key(p, &L[i]);
    qsort(L, (size_t)n, sizeof(leaf_t), cmp_leaf);
    orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
    m->p = *p;
    m->n = n;
    m->lev = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    m->g = (int64_t *)malloc(sizeof(int64_t) * 3 * (n > 0 ? n : 1));
    for (int i = 0; i < n; i++) {
        m->lev[i] = L[i].lev;
        for (int d = 0; d < 3; d++) m->g[3 * i + d] = L[i].g[d];
    }
    hash_build(m);
    return m;
}

/* Brick of trees refined uniformly to init_level (Sec. 2.2). */
orc_mesh *orc_mesh_new(const orc_params *p, int init_level)
{
    int64_t nb[3] = {1, 1, 1};
    for (int d = 0; d < p->ndim; d++) nb[d] = blocks_at(p, d, init_level);
    int n = (int)(nb[0] * nb[1] * nb[2]);
    leaf_t *L = (leaf_t *)calloc((size_t)n, sizeof(leaf_t));
    int c = 0;
    for (int64_t z = 0; z < nb[2]; z++)
        for (int64_t y = 0; y < nb[1]; y++)
            for (int64_t x = 0; x < nb[0]; x++) {
                L[c].lev = init_level;
                L[c].g[0] = x; L[c].g[1] = y; L[c].g[2] = z;
                c++;
            }
    orc_mesh *m = mesh_from_leaves(p, L, n);
    free(L);
    return m;
}

void orc_mesh_free(orc_mesh *m)
{
    if (!m) return;
    free(m->lev); free(m->g); free(m->hk); free(m->hv); free(m);
}

int orc_n_blocks(const orc_mesh *m) { return m->n; }

void orc_get_blocks(const orc_mesh *m, int32_t *lev, int64_t *g)
{
    for (int b = 0; b < m->n; b++) {
        lev[b] = m->lev[b];
        for (int d = 0; d < 3; d++) g[3 * b + d] = m->g[3 * b + d];
    }
}

/* ------------------------------------------------------------------------ */
/* Mesh adaptation: refine, coarsen, 2:1 balance with full connectivity      */
/* (Sec. 2.2: refine, coarsen, balance in that order; blocks sharing a       */
/* corner differ by at most one level).                                      */
/* ------------------------------------------------------------------------ */

/* Wrap or reject a block coordinate at level lev along dim d.
 * Returns 0 if outside a non-periodic domain. */
static int wrap_block(const orc_params *p, int d, int lev, int64_t *x)
{
    int64_t E = blocks_at(p, d, lev);
    if (*x >= 0 && *x < E) return 1;
    if (!p->periodic[d]) return 0;
    *x = ((*x % E) + E) % E;
    return 1;
}

/* Leaf containing the block-sized box (lev, g), searching levels lev..0;
 * returns -1 if the box is subdivided into finer leaves. */
static int leaf_covering_box(const orc_mesh *m, int lev, const int64_t g[3])
{
    for (int l = lev; l >= 0; l--) {
        int64_t a[3] = {0, 0, 0};
        for (int d = 0; d < m->p.ndim; d++) a[d] = g[d] >> (lev - l);
        int f = find_leaf(m, l, a);
        if (f >= 0) return f;
    }
    return -1;
}

static int push_children(const orc_params *p, leaf_t *out, int c, int lev, const int64_t g[3])
{
    int nc = 1 << p->ndim;
    for (int ch = 0; ch < nc; ch++) {
        out[c].lev = lev + 1;
        for (int d = 0; d < 3; d++)
            out[c].g[d] = (d < p->ndim) ? 2 * g[d] + ((ch >> d) & 1) : 0;
        c++;
    }
    return c;
}

/* flags: +1 refine, -1 coarsen, 0 keep (Sec. 2.2).  A family is coarsened only
 * when all of its 2^d children are leaves flagged -1; refinement stops at
 * max_level; balance only refines. */
orc_mesh *orc_adapt(const orc_mesh *m, const int8_t *flags)
{
    const orc_params *p = &m->p;
    int nc = 1 << p->ndim;
    int cap = m->n * nc + 16;
    leaf_t *L = (leaf_t *)calloc((size_t)cap, sizeof(leaf_t));
    int c = 0;
    /* parents whose family is coarsened, recorded once */
    uint64_t *done = (uint64_t *)calloc((size_t)m->n + 1, sizeof(uint64_t));
    int ndone = 0;
    for (int b = 0; b < m->n; b++) {
        const int64_t *g = &m->g[3 * b];
        int lev = m->lev[b];
        if (flags[b] > 0 && lev < p->max_level) {
            c = push_children(p, L, c, lev, g);
            continue;
        }
        if (flags[b] < 0 && lev > 0) {
            int64_t par[3] = {0, 0, 0};
            for (int d = 0; d < p->ndim; d++) par[d] = g[d] >> 1;
            int all = 1;
            for (int ch = 0; ch < nc && all; ch++) {
                int64_t s[3] = {0, 0, 0};
                for (int d = 0; d < p->ndim; d++) s[d] = 2 * par[d] + ((ch >> d) & 1);
                int f = find_leaf(m, lev, s);
                if (f < 0 || flags[f] >= 0) all = 0;
            }
            if (all) {
                uint64_t k = key_of(lev - 1, par);
                int seen = 0;
                for (int i = 0; i < ndone; i++) if (done[i] == k) { seen = 1; break; }
                if (!seen) {
                    done[ndone++] = k;
                    L[c].lev = lev - 1;
                    for (int d = 0; d < 3; d++) L[c].g[d] = par[d];
                    c++;
                }
                continue;
            }
        }
        L[c].lev = lev;
        for (int d = 0; d < 3; d++) L[c].g[d] = g[d];
        c++;
    }
    free(done);
    orc_mesh *cur = mesh_from_leaves(p, L, c);
    free(L);

    /* balance: repeat until no leaf has a corner/edge/face neighbour two or
     * more levels coarser */
    for (;;) {
        char *mark = (char *)calloc((size_t)cur->n, 1);
        int nmark = 0;
        int span[3] = {1, 1, 1};
        for (int d = 0; d < p->ndim; d++) span[d] = 3;
        for (int b = 0; b < cur->n; b++) {
            int lev = cur->lev[b];
            for (int dz = 0; dz < span[2]; dz++)
                for (int dy = 0; dy < span[1]; dy++)
                    for (int dx = 0; dx < span[0]; dx++) {
                        int off[3] = {dx - (span[0] > 1), dy - (span[1] > 1), dz - (span[2] > 1)};
                        if (!off[0] && !off[1] && !off[2]) continue;
                        int64_t q[3] = {0, 0, 0};
                        int inside = 1;
                        for (int d = 0; d < p->ndim; d++) {
                            q[d] = cur->g[3 * b + d] + off[d];
                            if (!wrap_block(p, d, lev, &q[d])) inside = 0;
                        }
                        if (!inside) continue;
                        int f = leaf_covering_box(cur, lev, q);
                        if (f >= 0 && cur->lev[f] <= lev - 2 && !mark[f]) { mark[f] = 1; nmark++; }
                    }
        }
        if (nmark == 0) { free(mark); break; }
        leaf_t *M = (leaf_t *)calloc((size_t)(cur->n * nc + 16), sizeof(leaf_t));
        int k = 0;
        for (int b = 0; b < cur->n; b++) {
            if (mark[b]) k = push_children(p, M, k, cur->lev[b], &cur->g[3 * b]);
            else { M[k].lev = cur->lev[b]; for (int d = 0; d < 3; d++) M[k].g[d] = cur->g[3 * b + d]; k++; }
        }
        free(mark);
        orc_mesh *nx = mesh_from_leaves(p, M, k);
        free(M);
        orc_mesh_free(cur);
        cur = nx;
    }
    return cur;
}

/* 1 if every pair of leaves sharing a face, edge or corner differs by at
 * most one level (checked by locating, for every leaf, all 3^d-1 same-size
 * neighbour boxes). */
int orc_check_balance(const orc_mesh *m)
{
    const orc_params *p = &m->p;
    int span[3] = {1, 1, 1};
    for (int d = 0; d < p->ndim; d++) span[d] = 3;
    for (int b = 0; b < m->n; b++) {
        int lev = m->lev[b];
        for (int dz = 0; dz < span[2]; dz++)
            for (int dy = 0; dy < span[1]; dy++)
                for (int dx = 0; dx < span[0]; dx++) {
                    int off[3] = {dx - (span[0] > 1), dy - (span[1] > 1), dz - (span[2] > 1)};
                    if (!off[0] && !off[1] && !off[2]) continue;
                    int64_t q[3] = {0, 0, 0};
                    int inside = 1;
                    for (int d = 0; d < p->ndim; d++) {
                        q[d] = m->g[3 * b + d] + off[d];
                        if (!wrap_block(p, d, lev, &q[d])) inside = 0;
                    }
                    if (!inside) continue;
                    int f = leaf_covering_box(m, lev, q);
                    if (f >= 0 && m->lev[f] <= lev - 2) return 0;
                }
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers                                                          */
/* ------------------------------------------------------------------------ */

static int SIDE(const orc_params *p) { return p->N + 2 * p->ng; }

static int64_t ncell(const orc_params *p)
{
    int64_t s = SIDE(p), c = 1;
    for (int d = 0; d < p->ndim; d++) c *= s;
    return c;
}

/* Flat offset of cell (i,j,k) (interior 0..N-1, ghosts outside) of variable v
 * of block b, layout uu(i,j,k,ivar,iblock) of Eq. 3 with i fastest. */
static int64_t at(const orc_params *p, int b, int v, int i, int j, int k)
{
    int64_t s = SIDE(p);
    int64_t c = (int64_t)(i + p->ng) + s * (int64_t)(j + p->ng);
    if (p->ndim == 3) c += s * s * (int64_t)(k + p->ng);
    return ((int64_t)b * p->nvar + v) * ncell(p) + c;
}

static int64_t atv(const orc_params *p, int b, int v, const int x[3])
{
    return at(p, b, v, x[0], x[1], p->ndim == 3 ? x[2] : 0);
}

static double dx_at(const orc_params *p, int d, int lev)
{
    return p->len[d] / (double)p->ntrees[d] / ((double)p->N * (double)(1LL << lev));
}

/* Leaf that holds the cell with global index C (at level lev, already
 * wrapped), searched at every level; *found_lev receives its level. */
static int locate_cell(const orc_mesh *m, int lev, const int64_t C[3], int *found_lev)
{
    const orc_params *p = &m->p;
    int hit = -1, nhit = 0;
    for (int l = 0; l <= p->max_level; l++) {
        int64_t bq[3] = {0, 0, 0};
        for (int d = 0; d < p->ndim; d++) {
            int64_t cl = (l >= lev) ? (C[d] << (l - lev)) : (C[d] >> (lev - l));
            bq[d] = cl / p->N;     /* cl >= 0 */
        }
        int f = find_leaf(m, l, bq);
        if (f >= 0) { hit = f; *found_lev = l; nhit++; }
    }
    return nhit == 1 ? hit : -1;
}

/* Global cell index of a block-local cell, wrapped; 0 when outside a
 * non-periodic domain. */
static int global_cell(const orc_mesh *m, int b, const int x[3], int64_t C[3])
{
    const orc_params *p = &m->p;
    int lev = m->lev[b];
    C[0] = C[1] = C[2] = 0;
    for (int d = 0; d < p->ndim; d++) {
        int64_t E = blocks_at(p, d, lev) * p->N;
        C[d] = m->g[3 * b + d] * p->N + x[d];
        if (C[d] < 0 || C[d] >= E) {
            if (!p->periodic[d]) return 0;
            C[d] = ((C[d] % E) + E) % E;
        }
    }
    return 1;
}

/* The lowest dimension in which block-local cell x lies outside block b
 * across a non-periodic domain boundary, or -1 if there is none. */
static int outside_dim(const orc_mesh *m, int b, const int x[3])
{
    const orc_params *p = &m->p;
    for (int d = 0; d < p->ndim; d++) {
        if (x[d] >= 0 && x[d] < p->N) continue;
        int64_t E = blocks_at(p, d, m->lev[b]);
        int64_t q = m->g[3 * b + d] + (x[d] < 0 ? -1 : 1);
        if (!p->periodic[d] && (q < 0 || q >= E)) return d;
    }
    return -1;
}

/* the tangential dimensions of face direction f, lower dimension first */
static void tangential(int ndim, int nd, int t[2])
{
    int c = 0;
    t[0] = t[1] = -1;
    for (int d = 0; d < ndim; d++) if (d != nd) t[c++] = d;
}

/* ------------------------------------------------------------------------ */
/* Ghost-cell pattern by brute force (Sec. 2.6): every ghost cell of every    */
/* face strip is located, and the strips are classified as SRL / F2C / C2F /  */
/* BC from the level of the leaf that holds them.                            */
/* Canonical export: one entry per (receiving block, face) -- per source      */
/* block for F2C -- with fields kind, face, dst, src, offset, aux, sorted by  */
/* (kind, face, dst, offset).  face = direction from dst towards src.  offset */
/* = position of the fine block inside the coarse face (bit 0: lower          */
/* tangential dim).  aux = boundary-face index for BC entries, else 0.        */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t kind, face, dst, src, offset, aux; } entry_t;

static int cmp_entry(const void *a, const void *b)
{
    const entry_t *x = (const entry_t *)a, *y = (const entry_t *)b;
    if (x->kind != y->kind) return x->kind < y->kind ? -1 : 1;
    if (x->face != y->face) return x->face < y->face ? -1 : 1;
    if (x->dst != y->dst) return x->dst < y->dst ? -1 : 1;
    if (x->offset != y->offset) return x->offset < y->offset ? -1 : 1;
    return 0;
}

/* Writes at most cap entries (6 int32 each) into out; returns the count, or
 * -1 if a strip mixes kinds / levels (2:1 balance broken). */
int64_t orc_pattern(const orc_mesh *m, int32_t *out, int64_t cap)
{
    const orc_params *p = &m->p;
    int N = p->N, ng = p->ng, D = p->ndim;
    int64_t maxe = (int64_t)m->n * (2 * D * (1 << (D - 1)) + 26) + 1;
    entry_t *E = (entry_t *)malloc(sizeof(entry_t) * maxe);
    int64_t ne = 0;
    int tn = (D == 3) ? N : 1;
    for (int b = 0; b < m->n; b++) {
        int lev = m->lev[b];
        for (int f = 0; f < 2 * D; f++) {
            int nd = f / 2, side = f % 2, td[2];
            tangential(D, nd, td);
            int nout = 0, ncell_s = 0;
            int srcs[8], nsrc = 0, slev = -100, mixed = 0;
            for (int kk = 1; kk <= ng; kk++)
                for (int t1 = 0; t1 < tn; t1++)
                    for (int t0 = 0; t0 < N; t0++) {
                        int x[3] = {0, 0, 0};
                        x[nd] = side ? N - 1 + kk : -kk;
                        x[td[0]] = t0;
                        if (D == 3) x[td[1]] = t1;
                        int64_t C[3];
                        ncell_s++;
                        if (!global_cell(m, b, x, C)) { nout++; continue; }
                        int fl;
                        int s = locate_cell(m, lev, C, &fl);
                        if (s < 0) { free(E); return -1; }
                        if (slev == -100) slev = fl;
                        else if (slev != fl) mixed = 1;
                        int seen = 0;
                        for (int i = 0; i < nsrc; i++) if (srcs[i] == s) seen = 1;
                        if (!seen) { if (nsrc == 8) { free(E); return -1; } srcs[nsrc++] = s; }
                    }
            if (nout) {
                if (nout != ncell_s) { free(E); return -1; }
                entry_t e = {K_BC, f, b, -1, 0, 0};
                E[ne++] = e;
                continue;
            }
            if (mixed) { free(E); return -1; }
            if (slev == lev) {
                if (nsrc != 1) { free(E); return -1; }
                entry_t e = {K_SRL, f, b, srcs[0], 0, 0};
                E[ne++] = e;
            } else if (slev == lev - 1) {
                if (nsrc != 1) { free(E); return -1; }
                int off = 0;
                for (int t = 0; t < D - 1; t++) off |= (int)(m->g[3 * b + td[t]] & 1) << t;
                entry_t e = {K_C2F, f, b, srcs[0], off, 0};
                E[ne++] = e;
            } else if (slev == lev + 1) {
                if (nsrc != (1 << (D - 1))) { free(E); return -1; }
                for (int i = 0; i < nsrc; i++) {
                    int s = srcs[i], off = 0;
                    for (int t = 0; t < D - 1; t++)
                        off |= (int)(m->g[3 * s + td[t]] - 2 * m->g[3 * b + td[t]]) << t;
                    entry_t e = {K_F2C, f, b, s, off, 0};
                    E[ne++] = e;
                }
            } else { free(E); return -1; }
        }
        /* edge and corner regions held by leaves of one level: a same-level
         * leaf (copy), a coarser leaf (prolongation, offset = parity of the
         * same-size box's coordinates, bit d for dimension d) or finer leaves
         * (restriction, one entry per fine leaf, offset = its position along
         * a 3D edge); a region reaching outside a non-periodic domain takes
         * the boundary formula of the face across its lowest such dimension
         * (offset = that face, aux = its boundary-face index) */
        if (p->diagonal) {
            for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); dz++)
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        int dir[3] = {dx, dy, dz};
                        int nz = (dx != 0) + (dy != 0) + (dz != 0);
                        if (nz < 2) continue;
                        int ok = 1, ext[3], lo[3], srcs[2], nsrc = 0, slev = -100;
                        int64_t C0[3] = {0, 0, 0};
                        for (int d = 0; d < 3; d++) {
                            lo[d] = dir[d] < 0 ? -ng : (dir[d] > 0 ? N : 0);
                            ext[d] = d >= D ? 1 : (dir[d] != 0 ? ng : N);
                            if (d >= D) lo[d] = 0;
                        }
                        int dout = outside_dim(m, b, lo);
                        if (dout >= 0) {
                            if (ne + 1 > maxe) { free(E); return -1; }
                            entry_t e = {K_DIAG_BC, diag_code(dir), b, -1, 2 * dout + (dir[dout] > 0), -1};
                            E[ne++] = e;
                            continue;
                        }
                        for (int k = 0; k < ext[2] && ok; k++)
                            for (int j = 0; j < ext[1] && ok; j++)
                                for (int i = 0; i < ext[0] && ok; i++) {
                                    int x[3] = {lo[0] + i, lo[1] + j, lo[2] + k};
                                    int64_t C[3];
                                    int fl;
                                    if (!global_cell(m, b, x, C)) { ok = 0; break; }
                                    int sblk = locate_cell(m, lev, C, &fl);
                                    if (sblk < 0 || fl < lev - 1 || fl > lev + 1) { ok = 0; break; }
                                    if (slev == -100) {
                                        slev = fl;
                                        for (int d = 0; d < 3; d++) C0[d] = C[d];
                                    } else if (slev != fl) { ok = 0; break; }
                                    int seen = 0;
                                    for (int q = 0; q < nsrc; q++) if (srcs[q] == sblk) seen = 1;
                                    if (!seen) {
                                        if (nsrc == 2) { ok = 0; break; }
                                        srcs[nsrc++] = sblk;
                                    }
                                }
                        if (!ok || nsrc == 0) continue;
                        if (ne + 2 > maxe) { free(E); return -1; }
                        if (slev == lev) {
                            if (nsrc != 1) continue;
                            entry_t e = {K_DIAG, diag_code(dir), b, srcs[0], 0, 0};
                            E[ne++] = e;
                        } else if (slev == lev - 1) {
                            if (nsrc != 1) continue;
                            int off = 0;
                            for (int d = 0; d < D; d++) off |= (int)((C0[d] / N) & 1) << d;
                            entry_t e = {K_DIAG_C2F, diag_code(dir), b, srcs[0], off, 0};
                            E[ne++] = e;
                        } else {
                            int ed = -1;     /* the edge dimension of a 3D edge */
                            for (int d = 0; d < D; d++) if (dir[d] == 0) ed = d;
                            for (int q = 0; q < nsrc; q++) {
                                int off = ed < 0 ? 0 : (int)(m->g[3 * srcs[q] + ed] - 2 * m->g[3 * b + ed]);
                                entry_t e = {K_DIAG_F2C, diag_code(dir), b, srcs[q], off, 0};
                                E[ne++] = e;
                            }
                        }
                    }
        }
    }
    qsort(E, (size_t)ne, sizeof(entry_t), cmp_entry);
    int32_t ibf = 0;
    for (int64_t i = 0; i < ne; i++) if (E[i].kind == K_BC) E[i].aux = ibf++;
    /* a boundary-formula edge or corner entry refers to its face's index */
    for (int64_t i = 0; i < ne; i++) {
        if (E[i].kind != K_DIAG_BC) continue;
        for (int64_t j = 0; j < ne; j++)
            if (E[j].kind == K_BC && E[j].dst == E[i].dst && E[j].face == E[i].offset) { E[i].aux = E[j].aux; break; }
    }
    int64_t w = ne < cap ? ne : cap;
    for (int64_t i = 0; i < w; i++) {
        out[6 * i + 0] = E[i].kind; out[6 * i + 1] = E[i].face; out[6 * i + 2] = E[i].dst;
        out[6 * i + 3] = E[i].src; out[6 * i + 4] = E[i].offset; out[6 * i + 5] = E[i].aux;
    }
    free(E);
    return ne;
}

/* Index of the boundary face (block b, face f) among all boundary faces in
 * the order (face direction, block), i.e. the order of the bc_data array
 * (Sec. 2.4, Eq. 4). */
static int boundary_face_index(const orc_mesh *m, int b, int f)
{
    const orc_params *p = &m->p;
    int idx = 0;
    for (int ff = 0; ff <= f; ff++) {
        int nd = ff / 2, side = ff % 2;
        if (p->periodic[nd]) continue;
        for (int bb = 0; bb < m->n; bb++) {
            if (ff == f && bb == b) return idx;
            int64_t E = blocks_at(p, nd, m->lev[bb]);
            int64_t gx = m->g[3 * bb + nd];
            if ((side == 0 && gx == 0) || (side == 1 && gx == E - 1)) idx++;
        }
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Restriction and limited prolongation (Sec. 2.2, Eq. 1 with theta = 1)     */
/* ------------------------------------------------------------------------ */

/* minmod: 0 unless both slopes have the same strict sign, else the one of
 * smaller magnitude (Eq. 1 with theta = 1). */
static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

/* Mean of the 2^d fine cells (fine index base[] .. base[]+1) of block fb,
 * summed as x-pairs, then y-pairs, then z-pairs. */
static double restrict_cell(const orc_params *p, const double *u, int fb, int v, const int base[3])
{
    double s[8];
    int D = p->ndim, n = 1 << D;
    for (int c = 0; c < n; c++) {
        int x[3] = {base[0] + (c & 1), base[1] + ((c >> 1) & 1), D == 3 ? base[2] + ((c >> 2) & 1) : 0};
        s[c] = u[atv(p, fb, v, x)];
    }
    /* pairwise: x, then y, then z */
    for (int w = n; w > 1; w /= 2)
        for (int c = 0; c < w / 2; c++) s[c] = s[2 * c] + s[2 * c + 1];
    return s[0] * (D == 3 ? 0.125 : 0.25);
}

/* Fine value inside coarse cell xc of block cb at sub-position sub[d] in
 * {0: lower half, 1: upper half}: u_c + (sum_d (+-1/4) G(u_c-u_{c-1}, u_{c+1}-u_c)). */
static double prolong_cell(const orc_params *p, const double *u, int cb, int v, const int xc[3], const int sub[3])
{
    double uc = u[atv(p, cb, v, xc)];
    double t = 0.0;
    for (int d = 0; d < p->ndim; d++) {
        int xm[3] = {xc[0], xc[1], xc[2]}, xp[3] = {xc[0], xc[1], xc[2]};
        xm[d] -= 1; xp[d] += 1;
        double slope = minmod(uc - u[atv(p, cb, v, xm)], u[atv(p, cb, v, xp)] - uc);
        double c = (sub[d] ? 0.25 : -0.25) * slope;
        t = (d == 0) ? c : t + c;
    }
    return uc + t;
}

/* ------------------------------------------------------------------------ */
/* Ghost fill, one cell at a time, in the two rounds of Sec. 2.6:             */
/*   R1: same level copies, physical boundaries, fine-to-coarse restriction;  */
/*   R2: coarse-to-fine limited prolongation (reads R1 ghosts).               */
/* Only face ghost cells are filled (Sec. 2.1: no edge or corner ghosts).     */
/* bc_data: [boundary face][var][N^(d-1)] Dirichlet values at face centres.   */
/* Returns 0, or -1 when a ghost cell has no valid source.                    */
/* ------------------------------------------------------------------------ */

static int fill_round(const orc_mesh *m, double *u, const double *bc_data, int round)
{
    const orc_params *p = &m->p;
    int N = p->N, ng = p->ng, D = p->ndim, V = p->nvar;
    int tn = (D == 3) ? N : 1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
    for (int b = 0; b < m->n; b++) {
        int lev = m->lev[b];
        for (int f = 0; f < 2 * D; f++) {
            int nd = f / 2, side = f % 2, td[2];
            tangential(D, nd, td);
            int ibf = -1;       /* boundary-face index, looked up once per face */
            for (int kk = 1; kk <= ng; kk++)
                for (int t1 = 0; t1 < tn; t1++)
                    for (int t0 = 0; t0 < N; t0++) {
                        int x[3] = {0, 0, 0};
                        x[nd] = side ? N - 1 + kk : -kk;
                        x[td[0]] = t0;
                        if (D == 3) x[td[1]] = t1;
                        int64_t C[3];
                        if (!global_cell(m, b, x, C)) {
                            if (round != 1) continue;
                            /* physical boundary (Sec. 2.4) */
                            int xm[3] = {x[0], x[1], x[2]};
                            xm[nd] = side ? N - kk : kk - 1;
                            int ty = p->bc_type[f];
                            double dxn = dx_at(p, nd, lev);
                            if (ty == BC_DATA && ibf < 0) ibf = boundary_face_index(m, b, f);
                            int64_t tt = t0 + (int64_t)N * t1;
                            int64_t nface = (D == 3) ? (int64_t)N * N : N;
                            for (int v = 0; v < V; v++) {
                                double um = u[atv(p, b, v, xm)], g;
                                if (ty == BC_DIRICHLET) g = 2.0 * p->bc_val[f][v] - um;
                                else if (ty == BC_NEUMANN) g = um + ((double)(2 * kk - 1) * dxn) * p->bc_val[f][v];
                                else if (ty == BC_DATA) g = 2.0 * bc_data[((int64_t)ibf * V + v) * nface + tt] - um;
                                else { err = 1; g = 0.0; }
                                u[atv(p, b, v, x)] = g;
                            }
                            continue;
                        }
                        int fl;
                        int s = locate_cell(m, lev, C, &fl);
                        if (s < 0 || fl < lev - 1 || fl > lev + 1) { err = 1; continue; }
                        if (fl == lev && round == 1) {
                            int xs[3] = {0, 0, 0};
                            for (int d = 0; d < D; d++) xs[d] = (int)(C[d] - m->g[3 * s + d] * N);
                            for (int v = 0; v < V; v++) u[atv(p, b, v, x)] = u[atv(p, s, v, xs)];
                        } else if (fl == lev + 1 && round == 1) {
                            int base[3] = {0, 0, 0};
                            for (int d = 0; d < D; d++) base[d] = (int)(2 * C[d] - m->g[3 * s + d] * N);
                            for (int v = 0; v < V; v++) u[atv(p, b, v, x)] = restrict_cell(p, u, s, v, base);
                        } else if (fl == lev - 1 && round == 2) {
                            int xc[3] = {0, 0, 0}, sub[3] = {0, 0, 0};
                            for (int d = 0; d < D; d++) {
                                xc[d] = (int)((C[d] >> 1) - m->g[3 * s + d] * N);
                                sub[d] = (int)(C[d] & 1);
                            }
                            for (int v = 0; v < V; v++) u[atv(p, b, v, x)] = prolong_cell(p, u, s, v, xc, sub);
                        }
                    }
        }
    }
    return err ? -1 : 0;
}

/* Edge and corner ghost cells (only when the mesh asks for them), one cell
 * at a time from the leaf that holds the cell's centre: round 1 copies from a
 * same-level leaf and restricts from a finer one, round 2 prolongs from a
 * coarser one (the limited prolongation reads the coarse leaf's interior and
 * round-1 face ghosts).  Cells outside a non-periodic domain are left to
 * fill_outside, which runs after both rounds. */
static void fill_diagonal(const orc_mesh *m, double *u, int round)
{
    const orc_params *p = &m->p;
    int N = p->N, ng = p->ng, D = p->ndim, V = p->nvar;
#pragma omp parallel for schedule(dynamic, 4)
    for (int b = 0; b < m->n; b++) {
        int lev = m->lev[b];
        int kr0 = (D == 3) ? -ng : 0, kr1 = (D == 3) ? N + ng : 1;
        for (int k = kr0; k < kr1; k++)
            for (int j = -ng; j < N + ng; j++)
                for (int i = -ng; i < N + ng; i++) {
                    int x[3] = {i, j, D == 3 ? k : 0};
                    int nout = 0;
                    for (int d = 0; d < D; d++) if (x[d] < 0 || x[d] >= N) nout++;
                    if (nout < 2) continue;
                    int64_t C[3];
                    int fl;
                    if (!global_cell(m, b, x, C)) continue;
                    int s = locate_cell(m, lev, C, &fl);
                    if (s < 0) continue;
                    if (fl == lev && round == 1) {
                        int xs[3] = {0, 0, 0};
                        for (int d = 0; d < D; d++) xs[d] = (int)(C[d] - m->g[3 * s + d] * N);
                        for (int v = 0; v < V; v++) u[atv(p, b, v, x)] = u[atv(p, s, v, xs)];
                    } else if (fl == lev + 1 && round == 1) {
                        int base[3] = {0, 0, 0};
                        for (int d = 0; d < D; d++) base[d] = (int)(2 * C[d] - m->g[3 * s + d] * N);
                        for (int v = 0; v < V; v++) u[atv(p, b, v, x)] = restrict_cell(p, u, s, v, base);
                    } else if (fl == lev - 1 && round == 2) {
                        int xc[3] = {0, 0, 0}, sub[3] = {0, 0, 0};
                        for (int d = 0; d < D; d++) {
                            xc[d] = (int)((C[d] >> 1) - m->g[3 * s + d] * N);
                            sub[d] = (int)(C[d] & 1);
                        }
                        for (int v = 0; v < V; v++) u[atv(p, b, v, x)] = prolong_cell(p, u, s, v, xc, sub);
                    }
                }
    }
}

/* Edge and corner ghost cells outside a non-periodic domain (only when the
 * mesh asks for edge and corner cells): each takes the boundary formula of
 * the face across its lowest dimension that leaves the domain, applied to
 * the cell mirrored across that face -- one dimension further in, so a face
 * ghost for an edge cell and an edge cell for a corner; edges are filled
 * before corners.  For per-cell boundary data the tangential position is
 * clamped to the face. */
static int fill_outside(const orc_mesh *m, double *u, const double *bc_data)
{
    const orc_params *p = &m->p;
    int N = p->N, ng = p->ng, D = p->ndim, V = p->nvar;
    int err = 0;
    for (int pass = 2; pass <= D; pass++) {
#pragma omp parallel for schedule(dynamic, 4) reduction(|| : err)
        for (int b = 0; b < m->n; b++) {
            int lev = m->lev[b];
            int kr0 = (D == 3) ? -ng : 0, kr1 = (D == 3) ? N + ng : 1;
            for (int k = kr0; k < kr1; k++)
                for (int j = -ng; j < N + ng; j++)
                    for (int i = -ng; i < N + ng; i++) {
                        int x[3] = {i, j, D == 3 ? k : 0};
                        int nout = 0;
                        for (int d = 0; d < D; d++) if (x[d] < 0 || x[d] >= N) nout++;
                        if (nout != pass) continue;
                        int d = outside_dim(m, b, x);
                        if (d < 0) continue;
                        int side = x[d] >= N ? 1 : 0, f = 2 * d + side;
                        int kk = side ? x[d] - N + 1 : -x[d];
                        int xm[3] = {x[0], x[1], x[2]};
                        xm[d] = side ? N - kk : kk - 1;
                        int ty = p->bc_type[f];
                        double dxn = dx_at(p, d, lev);
                        int td[2];
                        tangential(D, d, td);
                        int t0 = x[td[0]] < 0 ? 0 : (x[td[0]] >= N ? N - 1 : x[td[0]]);
                        int t1 = 0;
                        if (D == 3) t1 = x[td[1]] < 0 ? 0 : (x[td[1]] >= N ? N - 1 : x[td[1]]);
                        int64_t tt = t0 + (int64_t)N * t1;
                        int64_t nface = (D == 3) ? (int64_t)N * N : N;
                        int ibf = ty == BC_DATA ? boundary_face_index(m, b, f) : -1;
                        for (int v = 0; v < V; v++) {
                            double um = u[atv(p, b, v, xm)], g;
                            if (ty == BC_DIRICHLET) g = 2.0 * p->bc_val[f][v] - um;
                            else if (ty == BC_NEUMANN) g = um + ((double)(2 * kk - 1) * dxn) * p->bc_val[f][v];
                            else if (ty == BC_DATA) g = 2.0 * bc_data[((int64_t)ibf * V + v) * nface + tt] - um;
                            else { err = 1; g = 0.0; }
                            u[atv(p, b, v, x)] = g;
                        }
                    }
        }
    }
    return err ? -1 : 0;
}

int orc_fill_ghosts(const orc_mesh *m, double *u, const double *bc_data)
{
    if (fill_round(m, u, bc_data, 1)) return -1;
    if (m->p.diagonal) fill_diagonal(m, u, 1);
    if (fill_round(m, u, bc_data, 2)) return -1;
    if (m->p.diagonal) {
        fill_diagonal(m, u, 2);
        if (fill_outside(m, u, bc_data)) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Euler physics (Sec. 3.5, Eq. 14-16)                                        */
/* conservative U = (rho, rho v_0..v_{d-1}, E); primitive w = (rho, v, p)     */
/* ------------------------------------------------------------------------ */

static void to_primitive(int D, double gam, const double *U, double *w)
{
    double rho = U[0];
    double ke = 0.0;
    w[0] = rho;
    for (int d = 0; d < D; d++) {
        w[1 + d] = U[1 + d] / rho;
        ke = ke + w[1 + d] * w[1 + d];
    }
    ke = 0.5 * rho * ke;
    w[D + 1] = (gam - 1.0) * (U[D + 1] - ke);
}

static void to_conservative(int D, double gam, const double *w, double *U)
{
    double v2 = 0.0;
    U[0] = w[0];
    for (int d = 0; d < D; d++) {
        U[1 + d] = w[0] * w[1 + d];
        v2 = v2 + w[1 + d] * w[1 + d];
    }
    U[D + 1] = w[D + 1] / (gam - 1.0) + 0.5 * w[0] * v2;
}

/* physical flux along dimension n from primitive w */
static void phys_flux(int D, double gam, int n, const double *w, double *F)
{
    double U[5];
    to_conservative(D, gam, w, U);
    double vn = w[1 + n];
    F[0] = U[0] * vn;
    for (int d = 0; d < D; d++) F[1 + d] = U[1 + d] * vn + (d == n ? w[D + 1] : 0.0);
    F[D + 1] = (U[D + 1] + w[D + 1]) * vn;
}

/* Rusanov (local Lax-Friedrichs) flux with Einfeldt's wave-speed estimate
 * (Sec. 3.2 flux schemes; Sec. 3.5 wave speeds):
 *   u_roe = (sqrt(rL) uL + sqrt(rR) uR) / (sqrt(rL) + sqrt(rR))
 *   d^2   = (sqrt(rL) cL^2 + sqrt(rR) cR^2) / (sqrt(rL) + sqrt(rR))
 *           + 1/2 sqrt(rL) sqrt(rR) / (sqrt(rL) + sqrt(rR))^2 (uR - uL)^2
 *   a     = |u_roe| + d
 *   F     = (F(wL) + F(wR)) / 2 - a (U_R - U_L) / 2 */
static void rusanov(int D, double gam, int n, const double *wL, const double *wR, double *F)
{
    double FL[5], FR[5], UL[5], UR[5];
    phys_flux(D, gam, n, wL, FL);
    phys_flux(D, gam, n, wR, FR);
    to_conservative(D, gam, wL, UL);
    to_conservative(D, gam, wR, UR);
    double sL = sqrt(wL[0]), sR = sqrt(wR[0]);
    double cL2 = gam * wL[D + 1] / wL[0], cR2 = gam * wR[D + 1] / wR[0];
    double uL = wL[1 + n], uR = wR[1 + n];
    double inv = 1.0 / (sL + sR);
    double uroe = (sL * uL + sR * uR) * inv;
    double du = uR - uL;
    double d2 = (sL * cL2 + sR * cR2) * inv + 0.5 * sL * sR * inv * inv * du * du;
    double a = fabs(uroe) + sqrt(d2);
    for (int v = 0; v < D + 2; v++) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * a * (UR[v] - UL[v]);
}

/* HLL flux (Harten, Lax and van Leer) with the same Einfeldt estimates: the
 * smallest and largest signal speeds are u_roe -/+ d; with
 *   sL = min(u_roe - d, 0),  sR = max(u_roe + d, 0):
 *   F = (sR F(wL) - sL F(wR) + sL sR (U_R - U_L)) / (sR - sL),
 * which is F(wL) when all waves move right and F(wR) when all move left. */
static void hll(int D, double gam, int n, const double *wL, const double *wR, double *F)
{
    double FL[5], FR[5], UL[5], UR[5];
    phys_flux(D, gam, n, wL, FL);
    phys_flux(D, gam, n, wR, FR);
    to_conservative(D, gam, wL, UL);
    to_conservative(D, gam, wR, UR);
    double sqL = sqrt(wL[0]), sqR = sqrt(wR[0]);
    double cL2 = gam * wL[D + 1] / wL[0], cR2 = gam * wR[D + 1] / wR[0];
    double uL = wL[1 + n], uR = wR[1 + n];
    double inv = 1.0 / (sqL + sqR);
    double uroe = (sqL * uL + sqR * uR) * inv;
    double du = uR - uL;
    double d = sqrt((sqL * cL2 + sqR * cR2) * inv + 0.5 * sqL * sqR * inv * inv * du * du);
    double sL = uroe - d, sR = uroe + d;
    if (sL > 0.0) sL = 0.0;
    if (sR < 0.0) sR = 0.0;
    for (int v = 0; v < D + 2; v++) F[v] = (sR * FL[v] - sL * FR[v] + sL * sR * (UR[v] - UL[v])) / (sR - sL);
}

/* ------------------------------------------------------------------------ */
/* Scalar advection (Sec. 3.4, Eq. 13): d rho / dt + div(rho v) = 0 with a   */
/* uniform v.  Primitive and conservative variables are the same; along      */
/* dimension n the smallest and largest wave speeds are min(v_n, 0) and      */
/* max(v_n, 0), and the physical flux is rho v_n.  The two flux schemes of   */
/* Sec. 3.2 with those speeds:                                               */
/*   Rusanov: a = max(|min(v_n,0)|, |max(v_n,0)|) = |v_n|,                   */
/*            F = (rL v_n + rR v_n) / 2 - a (rR - rL) / 2                    */
/*   HLL:     sL = min(v_n,0), sR = max(v_n,0),                              */
/*            F = (sR rL v_n - sL rR v_n + sL sR (rR - rL)) / (sR - sL),     */
/*            and F = 0 when v_n = 0 (no wave, no flux).                     */
/* ------------------------------------------------------------------------ */

static void advection_flux(const orc_params *p, int n, double rL, double rR, double *F)
{
    double vn = p->velocity[n];
    double FL = rL * vn, FR = rR * vn;
    double sL = vn < 0.0 ? vn : 0.0;
    double sR = vn > 0.0 ? vn : 0.0;
    if (p->flux == 1) {
        if (sR - sL == 0.0) F[0] = 0.0;
        else F[0] = (sR * FL - sL * FR + sL * sR * (rR - rL)) / (sR - sL);
    } else {
        double a = fabs(sL) > fabs(sR) ? fabs(sL) : fabs(sR);
        F[0] = 0.5 * (FL + FR) - 0.5 * a * (rR - rL);
    }
}

static void face_flux(const orc_params *p, int n, const double *wL, const double *wR, double *F)
{
    if (p->physics == 1) advection_flux(p, n, wL[0], wR[0], F);
    else if (p->flux == 1) hll(p->ndim, p->gamma, n, wL, wR, F);
    else rusanov(p->ndim, p->gamma, n, wL, wR, F);
}

/* primitive variables of the configured physics (the identity for advection) */
static void primitive_of(const orc_params *p, const double *U, double *w)
{
    if (p->physics == 1) w[0] = U[0];
    else to_primitive(p->ndim, p->gamma, U, w);
}

/* a state the physics cannot hold: Euler with rho <= 0 or p <= 0 (the
 * advected scalar has no such bound) */
static int nonphysical(const orc_params *p, const double *w)
{
    if (p->physics == 1) return 0;
    return !(w[0] > 0.0) || !(w[p->ndim + 1] > 0.0);
}

/* Generalized minmod of the paper's Eq. 1: 0 when a and b differ in sign,
 * else sign(a) min(|theta a|, |theta b|, |a + b| / 2). */
static double gminmod(double a, double b, double theta)
{
    if (!((a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0))) return 0.0;
    double m = fabs(theta * a);
    if (fabs(theta * b) < m) m = fabs(theta * b);
    if (fabs(a + b) / 2.0 < m) m = fabs(a + b) / 2.0;
    return a > 0.0 ? m : -m;
}

/* Limited slope of a cell from its one-sided differences a (left) and b
 * (right), for the MUSCL face values w -/+ slope/2 (Sec. 3.2):
 *   0 minmod (Eq. 1, theta = 1); 1 monotonized central (Eq. 1, theta = 2);
 *   2 van Leer's harmonic mean 2ab / (a + b) when ab > 0, else 0. */
static double limited_slope(int lim, double a, double b)
{
    if (lim == 1) return gminmod(a, b, 2.0);
    if (lim == 2) return (a * b > 0.0) ? 2.0 * a * b / (a + b) : 0.0;
    return minmod(a, b);
}

/* WENO5 value at the face right of cell c from cells c-2 .. c+2 (Jiang & Shu
 * 1996): three third-order candidates q_k, smoothness indicators beta_k,
 * weights gamma = (1/10, 6/10, 3/10) / (eps + beta_k)^2 normalised, eps =
 * 1e-6.  The value at the face left of cell c is the same with the five
 * cells in reverse order. */
static double weno5(double a, double b, double c, double d, double e)
{
    double q0 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
    double q1 = (-b + 5.0 * c + 2.0 * d) / 6.0;
    double q2 = (2.0 * c + 5.0 * d - e) / 6.0;
    double t0 = a - 2.0 * b + c, u0 = a - 4.0 * b + 3.0 * c;
    double t1 = b - 2.0 * c + d, u1 = b - d;
    double t2 = c - 2.0 * d + e, u2 = 3.0 * c - 4.0 * d + e;
    double b0 = 13.0 / 12.0 * t0 * t0 + 0.25 * u0 * u0;
    double b1 = 13.0 / 12.0 * t1 * t1 + 0.25 * u1 * u1;
    double b2 = 13.0 / 12.0 * t2 * t2 + 0.25 * u2 * u2;
    const double eps = 1e-6;
    double a0 = 0.1 / ((eps + b0) * (eps + b0));
    double a1 = 0.6 / ((eps + b1) * (eps + b1));
    double a2 = 0.3 / ((eps + b2) * (eps + b2));
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/* Koren's limiter (Koren 1993), phi(r) = max(0, min(2r, (1 + 2r) / 3, 2)),
 * applied to the upwind difference: the face value right of a cell whose
 * left (upwind) and right differences are a and b is w + a phi(b / a) / 2,
 * and a phi(b / a) is 0 when ab <= 0, else sign(a) min(2|b|, (|a| + 2|b|) / 3,
 * 2|a|).  The face value left of the cell mirrors it: w - b phi(a / b) / 2. */
static double koren(double a, double b)
{
    if (!(a * b > 0.0)) return 0.0;
    double m = 2.0 * fabs(b);
    double t = (fabs(a) + 2.0 * fabs(b)) / 3.0;
    if (t < m) m = t;
    if (2.0 * fabs(a) < m) m = 2.0 * fabs(a);
    return a > 0.0 ? m : -m;
}

/* WENO3 value at the face right of cell c from cells c-1, c, c+1 (the
 * three-point member of the Jiang & Shu family): candidates q0 = -a/2 +
 * 3b/2 on {c-1, c} and q1 = (b + c)/2 on {c, c+1}, smoothness (b - a)^2 and
 * (c - b)^2, linear weights 1/3 and 2/3 over (eps + beta)^2, eps = 1e-6.  The
 * value at the face left of the cell takes the three cells in reverse order. */
static double weno3(double a, double b, double c)
{
    double q0 = -0.5 * a + 1.5 * b;
    double q1 = 0.5 * b + 0.5 * c;
    double b0 = (b - a) * (b - a), b1 = (c - b) * (c - b);
    const double eps = 1e-6;
    double a0 = (1.0 / 3.0) / ((eps + b0) * (eps + b0));
    double a1 = (2.0 / 3.0) / ((eps + b1) * (eps + b1));
    return (a0 * q0 + a1 * q1) / (a0 + a1);
}

/* The values of a cell w0 at its left (minus) and right (plus) faces along
 * one dimension from its neighbours wm, wp (Sec. 3.2 reconstruction with two
 * ghost layers): MUSCL w0 -/+ slope / 2 with the limited slope (minmod, MC,
 * van Leer), Koren's asymmetric limiter, WENO3, or first-order upwind
 * (the cell value itself, limiter 6). */
static void cell_faces(int lim, double wm, double w0, double wp, double *minus, double *plus)
{
    double a = w0 - wm, b = wp - w0;
    if (lim == 6) {
        *minus = w0;
        *plus = w0;
    } else if (lim == 4) {
        *plus = w0 + 0.5 * koren(a, b);
        *minus = w0 - 0.5 * koren(b, a);
    } else if (lim == 5) {
        *plus = weno3(wm, w0, wp);
        *minus = weno3(wp, w0, wm);
    } else {
        double s = 0.5 * limited_slope(lim, a, b);
        *plus = w0 + s;
        *minus = w0 - s;
    }
}

/* test hooks: the limiter and the face flux on given values */
double orc_limited_slope(int lim, double a, double b) { return limited_slope(lim, a, b); }
void orc_cell_faces(int lim, double wm, double w0, double wp, double *minus, double *plus) { cell_faces(lim, wm, w0, wp, minus, plus); }
double orc_weno5(double a, double b, double c, double d, double e) { return weno5(a, b, c, d, e); }
void orc_face_flux(const orc_params *p, int n, const double *wL, const double *wR, double *F) { face_flux(p, n, wL, wR, F); }

/* ------------------------------------------------------------------------ */
/* One forward-Euler sub-step of Eq. 5 (Sec. 3.1) with the finite-volume      */
/* steps of Sec. 3.2:                                                        */
/*   uo = dt_eff * F(ud) + sum_i w_i up_i                                    */
/* F: primitives on interior + face ghosts; MUSCL face values with the      */
/* limiter; Rusanov or HLL fluxes with Einfeldt speeds; divergence.  Then    */
/* flux fixing at refinement                                                 */
/* boundaries (Sec. 2.7): the coarse cells next to a face shared with finer  */
/* blocks get dt_eff/dx (F_coarse - mean F_fine) with the face's sign.        */
/* ud must have its face ghosts filled.  uo may alias one of up (each output  */
/* cell depends only on the same cell of up).                                */
/* Returns 0, or 1 when a non-physical state (rho <= 0 or p <= 0) was met.    */
/* ------------------------------------------------------------------------ */

int orc_stage(const orc_mesh *m, const double *ud, double *uo, int nprev,
              const double *const *up, const double *w, double dt_eff)
{
    const orc_params *p = &m->p;
    int N = p->N, D = p->ndim, V = p->nvar, S = SIDE(p);
    int64_t nc = ncell(p);
    int64_t nface = (D == 3) ? (int64_t)N * N : N;
    double gam = p->gamma;
    /* rhs for every block first, so that uo may alias up */
    double *rhs = (double *)calloc((size_t)m->n * V * nc, sizeof(double));
    /* boundary face fluxes: [block][face][var][N^(d-1)] */
    double *bf = (double *)calloc((size_t)m->n * 2 * D * V * nface, sizeof(double));
    int bad = 0;
    int tn = (D == 3) ? N : 1;

#pragma omp parallel for schedule(dynamic, 2) reduction(| : bad)
    for (int b = 0; b < m->n; b++) {
        double *wp = (double *)malloc(sizeof(double) * V * nc);
        int lev = m->lev[b];
        /* primitives on interior and face-ghost cells */
        int kr = (D == 3) ? S : 1;
        for (int kk = 0; kk < kr; kk++)
            for (int jj = 0; jj < S; jj++)
                for (int ii = 0; ii < S; ii++) {
                    int x[3] = {ii - p->ng, jj - p->ng, D == 3 ? kk - p->ng : 0};
                    int nout = 0;
                    for (int d = 0; d < D; d++) if (x[d] < 0 || x[d] >= N) nout++;
                    if (nout > 1) continue;
                    double U[5], W[5];
                    for (int v = 0; v < V; v++) U[v] = ud[atv(p, b, v, x)];
                    primitive_of(p, U, W);
                    if (nonphysical(p, W)) bad = 1;
                    int64_t c = (int64_t)ii + S * ((int64_t)jj + S * (int64_t)kk);
                    for (int v = 0; v < V; v++) wp[(int64_t)v * nc + c] = W[v];
                }
        /* face fluxes per dimension: fl[n][v][fp + (N+1)(t0 + N t1)], face fp
         * between cells fp-1 and fp along n */
        int64_t nfl = (int64_t)(N + 1) * nface;
        double *fl = (double *)malloc(sizeof(double) * D * V * nfl);
        for (int n = 0; n < D; n++) {
            int td[2];
            tangential(D, n, td);
            for (int t1 = 0; t1 < tn; t1++)
                for (int t0 = 0; t0 < N; t0++)
                    for (int fp = 0; fp <= N; fp++) {
                        double wm3[5], wm2[5], wm1[5], w0[5], w1[5], w2[5], wL[5], wR[5], F[5];
                        int weno = p->limiter == 3;
                        int pos[6] = {fp - 2, fp - 1, fp, fp + 1, fp - 3, fp + 2};
                        double *dst[6] = {wm2, wm1, w0, w1, wm3, w2};
                        for (int q = 0; q < (weno ? 6 : 4); q++) {
                            int x[3] = {0, 0, 0};
                            x[n] = pos[q]; x[td[0]] = t0;
                            if (D == 3) x[td[1]] = t1;
                            int64_t c = (int64_t)(x[0] + p->ng) + S * ((int64_t)(x[1] + p->ng) + (D == 3 ? S * (int64_t)(x[2] + p->ng) : 0));
                            for (int v = 0; v < V; v++) dst[q][v] = wp[(int64_t)v * nc + c];
                        }
                        /* reconstruction of primitives (Sec. 3.2): MUSCL with the
                         * limiter, or WENO5 from five cells on each side */
                        for (int v = 0; v < V; v++) {
                            if (weno) {
                                wL[v] = weno5(wm3[v], wm2[v], wm1[v], w0[v], w1[v]);
                                wR[v] = weno5(w2[v], w1[v], w0[v], wm1[v], wm2[v]);
                            } else {
                                double lo, hi;
                                cell_faces(p->limiter, wm2[v], wm1[v], w0[v], &lo, &hi);
                                wL[v] = hi;     /* right face of cell fp-1 */
                                cell_faces(p->limiter, wm1[v], w0[v], w1[v], &lo, &hi);
                                wR[v] = lo;     /* left face of cell fp */
                            }
                        }
                        if (nonphysical(p, wL) || nonphysical(p, wR)) bad = 1;
                        face_flux(p, n, wL, wR, F);
                        int64_t tt = t0 + (int64_t)N * t1;
                        for (int v = 0; v < V; v++) fl[((int64_t)n * V + v) * nfl + fp + (N + 1) * tt] = F[v];
                        if (fp == 0 || fp == N) {
                            int f = 2 * n + (fp == N);
                            for (int v = 0; v < V; v++)
                                bf[(((int64_t)b * 2 * D + f) * V + v) * nface + tt] = F[v];
                        }
                    }
        }
        /* divergence: rhs = sum_n (F_{n,lo} - F_{n,hi}) / dx_n, n = x first */
        int kr2 = (D == 3) ? N : 1;
        for (int k = 0; k < kr2; k++)
            for (int j = 0; j < N; j++)
                for (int i = 0; i < N; i++) {
                    int x[3] = {i, j, k};
                    for (int v = 0; v < V; v++) {
                        double r = 0.0;
                        for (int n = 0; n < D; n++) {
                            int td[2];
                            tangential(D, n, td);
                            int64_t tt = x[td[0]] + (int64_t)N * (D == 3 ? x[td[1]] : 0);
                            double Flo = fl[((int64_t)n * V + v) * nfl + x[n] + (N + 1) * tt];
                            double Fhi = fl[((int64_t)n * V + v) * nfl + x[n] + 1 + (N + 1) * tt];
                            r = r + (Flo - Fhi) / dx_at(p, n, lev);
                        }
                        /* gravity source S = (0, rho g, rho g.u) from the
                         * conservative state of the cell (Sec. 3.2 step order:
                         * source, then minus the flux divergence) */
                        if (p->physics == 1) {
                            /* advection: no source term */
                        } else if (v >= 1 && v <= D) {
                            r = r + ud[atv(p, b, 0, x)] * p->gravity[v - 1];
                        } else if (v == D + 1) {
                            double sg = 0.0;
                            for (int d = 0; d < D; d++) sg = sg + ud[atv(p, b, 1 + d, x)] * p->gravity[d];
                            r = r + sg;
                        }
                        rhs[atv(p, b, v, x)] = r;
                    }
                }
        free(fl);
        free(wp);
    }

    /* RK combination of Eq. 5 on interior cells */
#pragma omp parallel for schedule(static)
    for (int b = 0; b < m->n; b++) {
        int kr = (D == 3) ? N : 1;
        for (int v = 0; v < V; v++)
            for (int k = 0; k < kr; k++)
                for (int j = 0; j < N; j++)
                    for (int i = 0; i < N; i++) {
                        int64_t o = at(p, b, v, i, j, k);
                        double acc = 0.0;
                        for (int q = 0; q < nprev; q++) acc = (q == 0) ? w[0] * up[0][o] : acc + w[q] * up[q][o];
                        uo[o] = dt_eff * rhs[o] + acc;
                    }
    }

    /* flux fixing at refinement boundaries (Sec. 2.7), faces in order -x..+z */
    for (int b = 0; b < m->n; b++) {
        int lev = m->lev[b];
        for (int f = 0; f < 2 * D; f++) {
            int n = f / 2, side = f % 2, td[2];
            tangential(D, n, td);
            double dxn = dx_at(p, n, lev);
            for (int t1 = 0; t1 < tn; t1++)
                for (int t0 = 0; t0 < N; t0++) {
                    int x[3] = {0, 0, 0};
                    x[n] = side ? N : -1;        /* first cell across the face */
                    x[td[0]] = t0;
                    if (D == 3) x[td[1]] = t1;
                    int64_t C[3];
                    if (!global_cell(m, b, x, C)) continue;
                    int fl;
                    int s = locate_cell(m, lev, C, &fl);
                    if (s < 0 || fl != lev + 1) continue;
                    /* fine face cells covering this coarse face cell */
                    int64_t tt = t0 + (int64_t)N * t1;
                    int fo = 2 * n + (1 - side);   /* the fine block's face toward b */
                    double fsum[5][4];
                    int nf = 1 << (D - 1);
                    for (int a = 0; a < nf; a++) {
                        int64_t ft0 = 2 * C[td[0]] + (a & 1) - m->g[3 * s + td[0]] * N;
                        int64_t ft1 = (D == 3) ? 2 * C[td[1]] + ((a >> 1) & 1) - m->g[3 * s + td[1]] * N : 0;
                        int64_t ftt = ft0 + (int64_t)N * ft1;
                        for (int v = 0; v < V; v++)
                            fsum[v][a] = bf[(((int64_t)s * 2 * D + fo) * V + v) * nface + ftt];
                    }
                    int xi[3] = {0, 0, 0};
                    xi[n] = side ? N - 1 : 0;
                    xi[td[0]] = t0;
                    if (D == 3) xi[td[1]] = t1;
                    double q = dt_eff / dxn;
                    for (int v = 0; v < V; v++) {
                        double mean;
                        if (D == 3) mean = ((fsum[v][0] + fsum[v][1]) + (fsum[v][2] + fsum[v][3])) * 0.25;
                        else mean = (fsum[v][0] + fsum[v][1]) * 0.5;
                        double Fc = bf[(((int64_t)b * 2 * D + f) * V + v) * nface + tt];
                        double corr = q * (Fc - mean);
                        int64_t o = atv(p, b, v, xi);
                        uo[o] = side ? uo[o] + corr : uo[o] - corr;
                    }
                }
        }
    }
    free(rhs);
    free(bf);
    return bad;
}

/* ------------------------------------------------------------------------ */
/* CFL time-step limit (Sec. 3.2 step 2c): max over interior leaf cells of    */
/* sum_d (|v_d| + c) / dx_d, with c = sqrt(gamma p / rho) (Eq. 16); for      */
/* scalar advection sum_d |v_d| / dx_d with the uniform velocity.            */
/* dt = cfl / that maximum.                                                  */
/* ------------------------------------------------------------------------ */

double orc_max_speed(const orc_mesh *m, const double *u)
{
    const orc_params *p = &m->p;
    int N = p->N, D = p->ndim, V = p->nvar;
    double best = 0.0;
    for (int b = 0; b < m->n; b++) {
        int kr = (D == 3) ? N : 1;
        for (int k = 0; k < kr; k++)
            for (int j = 0; j < N; j++)
                for (int i = 0; i < N; i++) {
                    double s = 0.0;
                    if (p->physics == 1) {
                        /* advection: the wave speeds are those of v (Sec. 3.4) */
                        for (int d = 0; d < D; d++) s = s + fabs(p->velocity[d]) / dx_at(p, d, m->lev[b]);
                    } else {
                        double U[5], W[5];
                        for (int v = 0; v < V; v++) U[v] = u[at(p, b, v, i, j, k)];
                        to_primitive(D, p->gamma, U, W);
                        double c = sqrt(p->gamma * W[D + 1] / W[0]);
                        for (int d = 0; d < D; d++) s = s + (fabs(W[1 + d]) + c) / dx_at(p, d, m->lev[b]);
                    }
                    if (s > best) best = s;
                }
    }
    return best;
}

/* Integral of every conserved variable over the leaves (Eq. 18 summed over
 * the domain), accumulated in long double. */
void orc_conserved(const orc_mesh *m, const double *u, double *sums)
{
    const orc_params *p = &m->p;
    int N = p->N, D = p->ndim, V = p->nvar;
    for (int v = 0; v < V; v++) {
        long double acc = 0.0L;
        for (int b = 0; b < m->n; b++) {
            double vol = 1.0;
            for (int d = 0; d < D; d++) vol *= dx_at(p, d, m->lev[b]);
            int kr = (D == 3) ? N : 1;
            for (int k = 0; k < kr; k++)
                for (int j = 0; j < N; j++)
                    for (int i = 0; i < N; i++)
                        acc += (long double)u[at(p, b, v, i, j, k)] * (long double)vol;
        }
        sums[v] = (double)acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Refinement flags from the simplified Lohner estimator (Sec. 3.3, Eq. 12):   */
/*   E_n = |u_{n-1} - 2u_n + u_{n+1}| /                                      */
/*         (eps_abs + |u_n - u_{n-1}| + |u_{n+1} - u_n| + eps u*),             */
/*   u*  = |u_{n-1}| + 2|u_n| + |u_{n+1}|,  |E| = sqrt(sum_n E_n^2),          */
/* evaluated on density and pressure (on the scalar for advection); a cell's */
/* value is the larger of the                                                */
/* two.  +1 if some cell exceeds c_ref, -1 if every cell is below c_deref,    */
/* else 0.  u must have face ghosts filled.                                   */
/* ------------------------------------------------------------------------ */

static double lohner_1d(double um, double u0, double up, double eps, double eps_abs)
{
    double num = fabs(um - 2.0 * u0 + up);
    double ustar = fabs(um) + 2.0 * fabs(u0) + fabs(up);
    double den = eps_abs + fabs(u0 - um) + fabs(up - u0) + eps * ustar;
    return num / den;
}

void orc_lohner_flags(const orc_mesh *m, const double *u, double c_ref, double c_deref,
                      double eps, double eps_abs, int8_t *flags)
{
    const orc_params *p = &m->p;
    int N = p->N, D = p->ndim, V = p->nvar;
    for (int b = 0; b < m->n; b++) {
        int any_ref = 0, all_deref = 1;
        int kr = (D == 3) ? N : 1;
        for (int k = 0; k < kr; k++)
            for (int j = 0; j < N; j++)
                for (int i = 0; i < N; i++) {
                    double cellmax = 0.0;
                    for (int which = 0; which < 2; which++) {
                        double e2 = 0.0;
                        for (int n = 0; n < D; n++) {
                            double val[3];
                            for (int q = -1; q <= 1; q++) {
                                int x[3] = {i, j, k};
                                x[n] += q;
                                double U[5], W[5];
                                for (int v = 0; v < V; v++) U[v] = u[atv(p, b, v, x)];
                                primitive_of(p, U, W);
                                /* advection: the scalar stands in for both */
                                val[q + 1] = (which == 0 || p->physics == 1) ? W[0] : W[D + 1];
                            }
                            double e = lohner_1d(val[0], val[1], val[2], eps, eps_abs);
                            e2 = e2 + e * e;
                        }
                        double E = sqrt(e2);
                        if (E > cellmax) cellmax = E;
                    }
                    if (cellmax > c_ref) any_ref = 1;
                    if (!(cellmax < c_deref)) all_deref = 0;
                }
        flags[b] = any_ref ? 1 : (all_deref ? -1 : 0);
    }
}

/* The largest criterion value of each block (the quantity orc_lohner_flags
 * compares with c_ref and c_deref), computed by the same loops: per cell the
 * larger of the density and pressure values of |E|, per block the largest of
 * those.  Tests use it to put the thresholds exactly on a block's value. */
void orc_lohner_scores(const orc_mesh *m, const double *u, double eps, double eps_abs, double *scores)
{
    const orc_params *p = &m->p;
    int N = p->N, D = p->ndim, V = p->nvar;
    for (int b = 0; b < m->n; b++) {
        double bmax = 0.0;
        int kr = (D == 3) ? N : 1;
        for (int k = 0; k < kr; k++)
            for (int j = 0; j < N; j++)
                for (int i = 0; i < N; i++) {
                    double cellmax = 0.0;
                    for (int which = 0; which < 2; which++) {
                        double e2 = 0.0;
                        for (int n = 0; n < D; n++) {
                            double val[3];
                            for (int q = -1; q <= 1; q++) {
                                int x[3] = {i, j, k};
                                x[n] += q;
                                double U[5], W[5];
                                for (int v = 0; v < V; v++) U[v] = u[atv(p, b, v, x)];
                                primitive_of(p, U, W);
                                val[q + 1] = (which == 0 || p->physics == 1) ? W[0] : W[D + 1];
                            }
                            double e = lohner_1d(val[0], val[1], val[2], eps, eps_abs);
                            e2 = e2 + e * e;
                        }
                        double E = sqrt(e2);
                        if (E > cellmax) cellmax = E;
                    }
                    if (cellmax > bmax) bmax = cellmax;
                }
        scores[b] = bmax;
    }
}

/* ------------------------------------------------------------------------ */
/* Data transfer after a mesh change (Sec. 2.2): blocks that kept their level */
/* and position are copied; refined blocks are prolonged from the old parent  */
/* (limited prolongation, reading the parent's ghost cells at its edge);      */
/* coarsened blocks are restricted from the old children.  uold must have its */
/* face ghosts filled.  Only interior cells of unew are written.              */
/* Returns 0, or -1 if a new block changed by more than one level.            */
/* ------------------------------------------------------------------------ */

int orc_transfer(const orc_mesh *mo, const double *uold, const orc_mesh *mn, double *unew)
{
    const orc_params *p = &mn->p;
    int N = p->N, D = p->ndim, V = p->nvar;
    int kr = (D == 3) ? N : 1;
    for (int b = 0; b < mn->n; b++) {
        int lev = mn->lev[b];
        const int64_t *g = &mn->g[3 * b];
        int o = find_leaf(mo, lev, g);
        if (o >= 0) {
            for (int v = 0; v < V; v++)
                for (int k = 0; k < kr; k++)
                    for (int j = 0; j < N; j++)
                        for (int i = 0; i < N; i++)
                            unew[at(p, b, v, i, j, k)] = uold[at(p, o, v, i, j, k)];
            continue;
        }
        int64_t par[3] = {0, 0, 0};
        for (int d = 0; d < D; d++) par[d] = g[d] >> 1;
        o = (lev > 0) ? find_leaf(mo, lev - 1, par) : -1;
        if (o >= 0) {
            for (int v = 0; v < V; v++)
                for (int k = 0; k < kr; k++)
                    for (int j = 0; j < N; j++)
                        for (int i = 0; i < N; i++) {
                            int x[3] = {i, j, k}, xc[3] = {0, 0, 0}, sub[3] = {0, 0, 0};
                            for (int d = 0; d < D; d++) {
                                int64_t fine = (g[d] & 1) * N + x[d];
                                xc[d] = (int)(fine >> 1);
                                sub[d] = (int)(fine & 1);
                            }
                            unew[at(p, b, v, i, j, k)] = prolong_cell(p, uold, o, v, xc, sub);
                        }
            continue;
        }
        for (int k = 0; k < kr; k++)
            for (int j = 0; j < N; j++)
                for (int i = 0; i < N; i++) {
                    int x[3] = {i, j, k};
                    int64_t ch[3] = {0, 0, 0};
                    int base[3] = {0, 0, 0};
                    for (int d = 0; d < D; d++) {
                        int hi = x[d] >= N / 2;
                        ch[d] = 2 * g[d] + hi;
                        base[d] = 2 * (x[d] - hi * (N / 2));
                    }
                    int c = find_leaf(mo, lev + 1, ch);
                    if (c < 0) return -1;
                    for (int v = 0; v < V; v++)
                        unew[at(p, b, v, i, j, k)] = restrict_cell(p, uold, c, v, base);
                }
    }
    return 0;
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
