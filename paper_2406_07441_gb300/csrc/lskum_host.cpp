// Host side of liblskum: input validation, the colouring that fixes the
// LU-SGS sweep order (Alg. 5), the internal point order and neighbour layout,
// per-slot least-squares weights, device memory, one CUDA graph per
// iteration parity, and the C-ABI of include/lskum.h.
#include "lskum_internal.h"
#include "lskum_mlp_internal.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/lskum.h"
#include "../../include/lskum_mlp.h"

using namespace lskum;

namespace {

thread_local std::string g_create_error = "no error";

struct Arena {
    std::vector<void *> ptrs;
    cudaError_t err = cudaSuccess;
    template <class T>
    T *alloc(size_t count)
    {
        void *p = nullptr;
        if (err != cudaSuccess) return nullptr;
        err = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
        if (err != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    void release()
    {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

}  // namespace

struct lskum_ctx {
    int device = 0;
    int32_t n = 0, ld = 0;
    lskum_opts opts{};
    // host copies (caller order)
    std::vector<double> x, y, nx, ny;
    std::vector<uint8_t> flag;
    // order: internal position -> caller index, and the inverse
    std::vector<int32_t> perm, inv;
    std::vector<int32_t> colour;        // caller order, 1-based
    std::vector<int32_t> canon_order;   // stable colour order of caller indices
    int32_t n_colours = 0;
    int32_t n_levels = 0;               // sweep levels (colours, or (wall|interior, colour) pairs)
    std::vector<int32_t> lvl_beg, lvl_act_end, lvl_end;
    std::vector<int32_t> pk_lw[2];      // packed sweeps: first framed-point warp of each level (+ total), per direction
    std::vector<int32_t> lp_lg[2];      // packed sweeps: first interior group of each level (+ total), per direction
    bool pk_ok = false;                 // packed sweeps available (every list <= 32 slots)
    // device
    Arena arena;
    Dev dev{};
    Launch launch{};
    Ctrl *ctrl = nullptr;
    double *hist = nullptr, *hist4 = nullptr;
    int32_t hist_cap = 0;
    cudaStream_t stream = nullptr;      // internal, capture-capable
    cudaStream_t user_stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaStream_t side = nullptr;                      // side branch of the captured iterations
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    double *dscratch = nullptr;         // 4 * ld doubles on the device: caller-order staging
    bool host_direct_ok = false;        // the device reads and writes pageable host memory
    bool host_direct = false;           // host arrays go straight to / from the reorder kernels
    int launches_per_iter = 0;
    // cases (a batch is the disjoint union of its cases' clouds, caller order
    // = case 0's points, then case 1's, ...)
    int32_t n_cases = 1;
    std::vector<int32_t> case_off;      // [n_cases + 1] caller-order offsets
    std::vector<double> case_mach, case_aoa;
    std::vector<int32_t> case_of_caller;
    int32_t *case_state = nullptr, *case_it = nullptr;  // device, per case
    int32_t *case_err = nullptr, *case_bad = nullptr;
    double *case_hist0 = nullptr;
    // geometry the warm-start network reads (built on first use; internal order)
    float *mx = nullptr, *my = nullptr, *mdw = nullptr, *mcase_mach = nullptr, *mcase_aoa = nullptr;
    double *mcase_Uinf = nullptr, *mcase_uv = nullptr;
    int cur = 0;                        // state set holding the current state
    int64_t hist_bound = 0;             // upper bound of every case's recorded norms
    int cur_base = 0;
    bool pending = false;
    std::string err = "no error";
};

namespace {

// Conserved variables of a primitive state (Eq. 2); the one host formula for
// every state the library builds from primitives.
void host_prim_to_cons(double rho, double u, double v, double p, double *U)
{
    U[0] = rho;
    U[1] = rho * u;
    U[2] = rho * v;
    U[3] = p / 0.4 + 0.5 * rho * (u * u + v * v);
}

// Free-stream velocity of case b (the start state and the network's base).
void host_free_stream(const lskum_ctx *c, int32_t b, double *u, double *v)
{
    const double alb = c->case_aoa[b] * M_PI / 180.0;
    *u = c->case_mach[b] * std::cos(alb);
    *v = c->case_mach[b] * std::sin(alb);
}

lskum_status fail(lskum_ctx *c, lskum_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return s;
}

lskum_status cuda_fail(lskum_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, e == cudaErrorMemoryAllocation ? LSKUM_ERR_OOM : LSKUM_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// Greedy colouring of Alg. 5 on the symmetrised neighbour graph: each point's
// own stencil (given order) followed by the points that list it but are not
// in its stencil (ascending).  Visiting points in index order, every still
// uncoloured point (the visited one first, then its neighbours) receives the
// smallest colour > 0 not used by any of its neighbours.
// The other half of the symmetrised neighbour graph: for each point, the
// points that list it but are not in its own stencil, ascending (CSR).
void reverse_lists(int32_t n, const int32_t *off, const int32_t *idx, std::vector<int32_t> &rcnt,
                   std::vector<int32_t> &rev)
{
    rcnt.assign(n + 1, 0);
    auto listed_by = [&](int32_t q, int32_t p) {  // is p in stencil(q)?
        for (int32_t f = off[q]; f < off[q + 1]; f++)
            if (idx[f] == p) return true;
        return false;
    };
    for (int32_t p = 0; p < n; p++)
        for (int32_t e = off[p]; e < off[p + 1]; e++)
            if (!listed_by(idx[e], p)) rcnt[idx[e] + 1]++;
    for (int32_t p = 0; p < n; p++) rcnt[p + 1] += rcnt[p];
    rev.assign(std::max<int32_t>(rcnt[n], 1), 0);
    std::vector<int32_t> fill(n, 0);
    for (int32_t p = 0; p < n; p++)
        for (int32_t e = off[p]; e < off[p + 1]; e++) {
            const int32_t q = idx[e];
            if (!listed_by(q, p)) rev[rcnt[q] + fill[q]++] = p;
        }
}

int32_t colour_points(int32_t n, const int32_t *off, const int32_t *idx, std::vector<int32_t> &col)
{
    std::vector<int32_t> rcnt, rev;
    reverse_lists(n, off, idx, rcnt, rev);
    col.assign(n, 0);
    std::vector<int32_t> seen;  // seen[colour] == stamp when used by a neighbour
    int32_t stamp = 0;
    auto smallest = [&](int32_t p) {
        stamp++;
        auto mark = [&](int32_t q) {
            const int32_t cq = col[q];
            if (cq >= (int32_t)seen.size()) seen.resize(cq + 1, 0);
            seen[cq] = stamp;
        };
        for (int32_t f = off[p]; f < off[p + 1]; f++) mark(idx[f]);
        for (int32_t f = rcnt[p]; f < rcnt[p + 1]; f++) mark(rev[f]);
        int32_t k = 1;
        while (k < (int32_t)seen.size() && seen[k] == stamp) k++;
        return k;
    };
    if (n > 0) col[0] = 1;
    for (int32_t i = 0; i < n; i++) {
        if (col[i] == 0) col[i] = smallest(i);
        for (int32_t f = off[i]; f < off[i + 1]; f++)
            if (col[idx[f]] == 0) col[idx[f]] = smallest(idx[f]);
        for (int32_t f = rcnt[i]; f < rcnt[i + 1]; f++)
            if (col[rev[f]] == 0) col[rev[f]] = smallest(rev[f]);
    }
    int32_t nc = 0;
    for (int32_t p = 0; p < n; p++) nc = std::max(nc, col[p]);
    return nc;
}

}  // namespace

extern "C" {

const char *lskum_last_error(const lskum_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

// Host-side arrays of the internal layout, built before any device call.
struct HostPrep {
    std::vector<int32_t> slice_off, deg, enb;
    std::vector<uint8_t> emb, fl_i;
    std::vector<double> edx, edy, ew1, ew2, egx, egy, geo_i, wnx, wny;
    std::vector<double> exx, exy, eyx, eyy;  // wgx dx, wgx dy, wgy dx, wgy dy per slot
    // LU-SGS lower / upper slot lists (CSR, internal order) and level orders
    std::vector<int32_t> lo_off, lo_nbr, up_off, up_nbr, sw_fwd, sw_bwd;
    std::vector<uint8_t> lo_mb, up_mb;
    std::vector<double> lo_w1, lo_w2, up_w1, up_w2;
    // per-case norm blocks and case of every internal point
    std::vector<int32_t> blk_pos, blk_case, case_blk, case_of_i;
    std::vector<uint8_t> smb_caller;  // sub-stencil membership per caller-order slot
    // packed sweep form per direction (0 forward / lower lists, 1 backward / upper lists)
    std::vector<int32_t> pk_pt[2], pk_nbr[2];
    std::vector<uint8_t> pk_mb[2], pk_steps[2];
    std::vector<double> pk_w1[2], pk_w2[2];
    // interior points in lane-per-point groups of 32 (thread t of group g:
    // point lp_k[32 g + t], -1 for none, with lp_len[32 g + t] slots at
    // lp_goff[g] + 32 j + t)
    std::vector<int32_t> lp_k[2], lp_len[2], lp_goff[2], lp_nbr[2];
    std::vector<uint8_t> lp_mb[2];
    std::vector<double> lp_w1[2], lp_w2[2];
};
static lskum_status prepare_host(lskum_ctx *c, const lskum_cloud *cl, HostPrep &hp);

// Is point p (caller order of the union) an unknown of the iteration?  Outer
// points are only under the kinetic far field.
static bool swept(const lskum_ctx *c, int32_t p)
{
    return c->flag[p] != LSKUM_OUTER || c->opts.farfield == LSKUM_FARFIELD_KINETIC;
}
static lskum_status upload(lskum_ctx *c, HostPrep &hp);
static lskum_status build_graphs(lskum_ctx *c);

static bool opts_valid(const lskum_opts *o)
{
    return (o->cfl > 0.0) && std::isfinite(o->cfl) && std::isfinite(o->mach) && std::isfinite(o->aoa_deg) &&
           (o->cfl_ramp_iters >= 0.0) && o->inner_iters >= 0 && o->inner_iters <= 64 &&
           (o->jvp == LSKUM_JVP_EXACT || o->jvp == LSKUM_JVP_INCREMENT) && (o->precision == 0 || o->precision == 1) &&
           o->first_order_iters >= 0 &&
           (o->scheme == LSKUM_SCHEME_LUSGS || (o->scheme == LSKUM_SCHEME_EXPLICIT && o->precision == 0)) &&
           (o->lusgs == LSKUM_LUSGS_ANANDH || o->lusgs == LSKUM_LUSGS_MANISH) &&
           (o->ordering == LSKUM_ORDER_COLOUR || o->ordering == LSKUM_ORDER_WALL_FIRST ||
            o->ordering == LSKUM_ORDER_SERIAL) &&
           (o->farfield == LSKUM_FARFIELD_FREESTREAM || o->farfield == LSKUM_FARFIELD_KINETIC);
}

static bool opts_shared_equal(const lskum_opts *a, const lskum_opts *b)
{
    return a->cfl == b->cfl && a->cfl_ramp_iters == b->cfl_ramp_iters && a->inner_iters == b->inner_iters &&
           a->jvp == b->jvp && a->precision == b->precision && a->first_order_iters == b->first_order_iters &&
           a->scheme == b->scheme && a->lusgs == b->lusgs && a->ordering == b->ordering && a->farfield == b->farfield;
}

// Validate one case's cloud (indices local to the case); `kinetic`: outer
// points need outward unit normals (the kinetic far field).
static lskum_status validate_cloud(const lskum_cloud *cl, int32_t cs, bool kinetic)
{
    if (!cl) return fail(nullptr, LSKUM_ERR_ARG, "case %d: cloud is NULL", cs);
    const int32_t n = cl->n_points;
    if (n < 1) return fail(nullptr, LSKUM_ERR_ARG, "case %d: n_points = %d < 1", cs, n);
    if (!cl->x || !cl->y || !cl->flag || !cl->nbr_off || !cl->nbr_idx)
        return fail(nullptr, LSKUM_ERR_ARG, "case %d: a cloud array is NULL", cs);
    const int32_t *off = cl->nbr_off, *idx = cl->nbr_idx;
    if (off[0] != 0) return fail(nullptr, LSKUM_ERR_ARG, "case %d: nbr_off[0] != 0", cs);
    bool has_wall = false, has_outer = false;
    for (int32_t p = 0; p < n; p++) {
        if (off[p + 1] < off[p]) return fail(nullptr, LSKUM_ERR_ARG, "nbr_off decreases at point %d", p);
        if (cl->flag[p] > LSKUM_OUTER) return fail(nullptr, LSKUM_ERR_ARG, "bad flag at point %d", p);
        if (!std::isfinite(cl->x[p]) || !std::isfinite(cl->y[p]))
            return fail(nullptr, LSKUM_ERR_ARG, "non-finite coordinate at point %d", p);
        if (off[p + 1] - off[p] > 255) return fail(nullptr, LSKUM_ERR_ARG, "more than 255 neighbours at point %d", p);
        has_wall |= cl->flag[p] == LSKUM_WALL;
        has_outer |= cl->flag[p] == LSKUM_OUTER;
    }
    if (!cl->nx != !cl->ny) return fail(nullptr, LSKUM_ERR_ARG, "case %d: nx and ny must both be given or both NULL", cs);
    for (int32_t p = 0; p < n; p++) {
        for (int32_t e = off[p]; e < off[p + 1]; e++) {
            const int32_t q = idx[e];
            if (q < 0 || q >= n || q == p)
                return fail(nullptr, LSKUM_ERR_ARG, "bad neighbour index %d at point %d", q, p);
            for (int32_t f = off[p]; f < e; f++)
                if (idx[f] == q) return fail(nullptr, LSKUM_ERR_ARG, "duplicate neighbour %d at point %d", q, p);
        }
        if (cl->nx && (cl->flag[p] == LSKUM_WALL || (kinetic && cl->flag[p] == LSKUM_OUTER))) {
            const double ln = std::hypot(cl->nx[p], cl->ny[p]);
            if (!(std::fabs(ln - 1.0) < 1e-6))
                return fail(nullptr, LSKUM_ERR_ARG, "%s normal not unit at point %d",
                            cl->flag[p] == LSKUM_WALL ? "wall" : "outer", p);
        }
    }
    return LSKUM_OK;
}

// Unit normals of the closed polygon of a case's points of type `type`, in
// caller order: the central-difference tangent (next - previous) rotated to
// its right, turned so that it points away from the region the polygon
// encloses when that region is the body (wall) and out of the domain for the
// outer boundary -- both the right-hand normal of a counter-clockwise polygon.
// Errors: fewer than 3 such points, or a zero tangent.
static lskum_status polygon_normals(const lskum_cloud *cl, int32_t cs, uint8_t type, double *nx, double *ny)
{
    std::vector<int32_t> v;
    for (int32_t p = 0; p < cl->n_points; p++)
        if (cl->flag[p] == type) v.push_back(p);
    if (v.empty()) return LSKUM_OK;
    const size_t m = v.size();
    if (m < 3) return fail(nullptr, LSKUM_ERR_ARG, "case %d: fewer than 3 %s points to form a polygon", cs,
                           type == LSKUM_WALL ? "wall" : "outer");
    double area2 = 0.0;
    for (size_t k = 0; k < m; k++) {
        const int32_t a = v[k], b = v[(k + 1) % m];
        area2 += cl->x[a] * cl->y[b] - cl->x[b] * cl->y[a];
    }
    const double orient = area2 > 0.0 ? 1.0 : -1.0;
    for (size_t k = 0; k < m; k++) {
        const int32_t a = v[(k + m - 1) % m], p = v[k], b = v[(k + 1) % m];
        const double tx = cl->x[b] - cl->x[a], ty = cl->y[b] - cl->y[a];
        const double ln = std::hypot(tx, ty);
        if (!(ln > 0.0)) return fail(nullptr, LSKUM_ERR_ARG, "case %d: zero polygon tangent at point %d", cs, p);
        nx[p] = orient * ty / ln;
        ny[p] = -orient * tx / ln;
    }
    return LSKUM_OK;
}

// Invariants of the host layout that the kernels rely on: the internal order
// is a permutation, every wall or interior point (and, under the kinetic far
// field, every outer point) lies in exactly one sweep level and frozen outer
// points in none, each level's two sweep orders are
// permutations of the level, no two points of a level are coupled, and
// every lower (upper) slot list entry lies in an earlier (later) level, the
// two lists together holding every coupling slot.
static lskum_status verify_layout(lskum_ctx *c, const lskum_cloud *cl, const HostPrep &hp)
{
    const int32_t n = c->n;
    std::vector<int32_t> seen(n, 0);
    for (int32_t k = 0; k < n; k++) {
        const int32_t p = c->perm[k];
        if (p < 0 || p >= n || seen[p]++ || c->inv[p] != k) return fail(c, LSKUM_ERR_ARG, "layout: order");
    }
    std::vector<int32_t> level(n, -1);
    int32_t prev_end = 0;
    for (int32_t l = 0; l < c->n_levels; l++) {
        const int32_t b = c->lvl_beg[l], ae = c->lvl_act_end[l], e = c->lvl_end[l];
        if (!(b >= prev_end && b < ae && ae <= e && e <= n)) return fail(c, LSKUM_ERR_ARG, "layout: level %d", l);
        prev_end = e;
        std::vector<int32_t> f(hp.sw_fwd.begin() + b, hp.sw_fwd.begin() + ae),
            g(hp.sw_bwd.begin() + b, hp.sw_bwd.begin() + ae);
        std::sort(f.begin(), f.end());
        std::sort(g.begin(), g.end());
        for (int32_t k = b; k < ae; k++) {
            if (f[k - b] != k || g[k - b] != k) return fail(c, LSKUM_ERR_ARG, "layout: sweep order of level %d", l);
            if (!swept(c, c->perm[k])) return fail(c, LSKUM_ERR_ARG, "layout: frozen outer point swept");
            level[k] = l;
        }
    }
    for (int32_t k = 0; k < n; k++)
        if ((level[k] < 0) == swept(c, c->perm[k]))
            return fail(c, LSKUM_ERR_ARG, "layout: point %d not in a level", c->perm[k]);
    for (int32_t k = 0; k < n; k++) {
        if (level[k] < 0) continue;
        int32_t coupled = 0;
        const int32_t p = c->perm[k];
        for (int32_t e = cl->nbr_off[p]; e < cl->nbr_off[p + 1]; e++) {
            const int32_t q = c->inv[cl->nbr_idx[e]];
            if (level[q] < 0) continue;
            if (level[q] == level[k]) return fail(c, LSKUM_ERR_ARG, "layout: coupled points %d, %d in one level", p,
                                                  cl->nbr_idx[e]);
        }
        for (int32_t j = hp.lo_off[k]; j < hp.lo_off[k + 1]; j++, coupled++)
            if (hp.lo_nbr[j] < 0 || hp.lo_nbr[j] >= n || !(level[hp.lo_nbr[j]] >= 0 && level[hp.lo_nbr[j]] < level[k]))
                return fail(c, LSKUM_ERR_ARG, "layout: lower list of point %d", p);
        for (int32_t j = hp.up_off[k]; j < hp.up_off[k + 1]; j++, coupled++)
            if (hp.up_nbr[j] < 0 || hp.up_nbr[j] >= n || !(level[hp.up_nbr[j]] > level[k]))
                return fail(c, LSKUM_ERR_ARG, "layout: upper list of point %d", p);
        int32_t expect = 0;
        for (int32_t e = cl->nbr_off[p]; e < cl->nbr_off[p + 1]; e++)
            expect += level[c->inv[cl->nbr_idx[e]]] >= 0 && hp.smb_caller[e] != 0;
        if (coupled != expect) return fail(c, LSKUM_ERR_ARG, "layout: slot lists of point %d", p);
    }
    for (int64_t t = 0; t < (int64_t)hp.enb.size(); t++)
        if (hp.enb[t] < 0 || hp.enb[t] >= n) return fail(c, LSKUM_ERR_ARG, "layout: neighbour slot");
    // packed sweep form: each level's warps hold exactly its points, each
    // point's list (or one empty slot) in consecutive lanes of one warp
    for (int dir = 0; dir < 2 && c->pk_ok; dir++) {
        const std::vector<int32_t> &lw = c->pk_lw[dir], &pt = hp.pk_pt[dir], &nb = hp.pk_nbr[dir];
        const std::vector<int32_t> &so = dir == 0 ? hp.sw_fwd : hp.sw_bwd;
        const std::vector<int32_t> &loff = dir == 0 ? hp.lo_off : hp.up_off;
        const std::vector<int32_t> &lnbr = dir == 0 ? hp.lo_nbr : hp.up_nbr;
        if ((int32_t)lw.size() != c->n_levels + 1 || (size_t)lw.back() * 32 != pt.size() || nb.size() != pt.size() ||
            hp.pk_steps[dir].size() != (size_t)lw.back())
            return fail(c, LSKUM_ERR_ARG, "layout: packed sweep size");
        for (int64_t w = 0; w < lw.back(); w++) {  // each segment fits the warp's sum steps
            int32_t run = 0;
            for (int64_t t = w * 32; t < w * 32 + 32; t++) {
                run = (t > w * 32 && pt[t] == pt[t - 1] && pt[t] >= 0) ? run + 1 : 1;
                if (pt[t] >= 0 && run > (1 << hp.pk_steps[dir][w]))
                    return fail(c, LSKUM_ERR_ARG, "layout: packed sum steps of warp %lld", (long long)w);
            }
        }
        // interior groups: sizes, and every lane's list inside its group's slots
        const std::vector<int32_t> &lg = c->lp_lg[dir], &lk = hp.lp_k[dir], &ll = hp.lp_len[dir];
        const std::vector<int32_t> &go = hp.lp_goff[dir], &lnb = hp.lp_nbr[dir];
        if ((int32_t)lg.size() != c->n_levels + 1 || lg[0] != 0 || (size_t)lg.back() * kPointsPerWarp != lk.size() ||
            ll.size() != lk.size() || go.size() != (size_t)lg.back() + 1 || go[0] != 0 ||
            (size_t)go.back() != lnb.size() || hp.lp_mb[dir].size() != lnb.size() ||
            hp.lp_w1[dir].size() != lnb.size() || hp.lp_w2[dir].size() != lnb.size())
            return fail(c, LSKUM_ERR_ARG, "layout: interior groups size");
        std::vector<int32_t> pos_of(n, -1);  // sweep position of each swept point
        for (int32_t l = 0; l < c->n_levels; l++)
            for (int32_t pos = c->lvl_beg[l]; pos < c->lvl_act_end[l]; pos++)
                if (so[pos] >= 0 && so[pos] < n) pos_of[so[pos]] = pos;
        std::vector<int32_t> seen_pos(n, 0);
        for (int32_t l = 0; l < c->n_levels; l++) {
            for (int64_t t = (int64_t)lw[l] * 32; t < (int64_t)lw[l + 1] * 32; t++) {
                const int32_t pos = pt[t];
                if (pos < 0) continue;
                if (pos < c->lvl_beg[l] || pos >= c->lvl_act_end[l] || nb[t] < 0 || nb[t] >= n)
                    return fail(c, LSKUM_ERR_ARG, "layout: packed slot %lld", (long long)t);
                if (t % 32 != 0 && pt[t - 1] == pos) continue;  // not the point's first slot
                if (seen_pos[pos]++) return fail(c, LSKUM_ERR_ARG, "layout: packed point split");
                const int32_t k = so[pos], len = loff[k + 1] - loff[k];
                if (t % 32 + std::max(1, len) > 32) return fail(c, LSKUM_ERR_ARG, "layout: packed point crosses a warp");
                for (int32_t j = 0; j < std::max(1, len); j++)
                    if (pt[t + j] != pos || (len > 0 && nb[t + j] != lnbr[loff[k] + j]))
                        return fail(c, LSKUM_ERR_ARG, "layout: packed list of position %d", pos);
                if (t % 32 + std::max(1, len) < 32 && pt[t + std::max(1, len)] == pos)
                    return fail(c, LSKUM_ERR_ARG, "layout: packed list of position %d too long", pos);
            }
            if (lg[l + 1] < lg[l]) return fail(c, LSKUM_ERR_ARG, "layout: interior groups of level %d", l);
            for (int64_t g = lg[l]; g < lg[l + 1]; g++) {
                if (go[g + 1] < go[g] || (go[g + 1] - go[g]) % 32 != 0)
                    return fail(c, LSKUM_ERR_ARG, "layout: interior group %lld", (long long)g);
                const int32_t width = (go[g + 1] - go[g]) / 32;
                constexpr int L = kLanesPerPoint;
                for (int32_t t = 0; t < kPointsPerWarp; t++) {
                    const int32_t k = lk[(int64_t)kPointsPerWarp * g + t];
                    if (k < 0) continue;
                    if (k >= n || c->flag[c->perm[k]] != LSKUM_INTERIOR)
                        return fail(c, LSKUM_ERR_ARG, "layout: interior group %lld", (long long)g);
                    const int32_t pos = pos_of[k], len = loff[k + 1] - loff[k];
                    if (pos < c->lvl_beg[l] || pos >= c->lvl_act_end[l] || seen_pos[pos]++)
                        return fail(c, LSKUM_ERR_ARG, "layout: interior point %d", k);
                    if (ll[(int64_t)kPointsPerWarp * g + t] != len || (len + L - 1) / L > width)
                        return fail(c, LSKUM_ERR_ARG, "layout: interior list of point %d", k);
                    for (int32_t j = 0; j < len; j++) {
                        const int64_t e = go[g] + 32 * (int64_t)(j / L) + L * t + j % L;
                        if (lnb[e] != lnbr[loff[k] + j] || lnb[e] < 0 || lnb[e] >= n)
                            return fail(c, LSKUM_ERR_ARG, "layout: interior list of point %d", k);
                    }
                }
            }
            for (int32_t pos = c->lvl_beg[l]; pos < c->lvl_act_end[l]; pos++)
                if (seen_pos[pos] != 1) return fail(c, LSKUM_ERR_ARG, "layout: position %d not packed", pos);
        }
    }
    return LSKUM_OK;
}

static lskum_status create_impl(const lskum_cloud *clouds, const lskum_opts *opts, int32_t n_cases,
                                void *cuda_stream, lskum_ctx **out, bool host_only = false,
                                int32_t *n_colours = nullptr, int32_t *n_levels = nullptr)
{
    if (!out) return fail(nullptr, LSKUM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!clouds || !opts || n_cases < 1) return fail(nullptr, LSKUM_ERR_ARG, "clouds, opts or n_cases invalid");
    int64_t total = 0, total_nnz = 0;
    for (int32_t b = 0; b < n_cases; b++) {
        if (!opts_valid(&opts[b])) return fail(nullptr, LSKUM_ERR_ARG, "invalid option value (case %d)", b);
        if (!opts_shared_equal(&opts[0], &opts[b]))
            return fail(nullptr, LSKUM_ERR_ARG, "case %d: options other than mach/aoa differ from case 0", b);
        lskum_status v = validate_cloud(&clouds[b], b, opts[0].farfield == LSKUM_FARFIELD_KINETIC);
        if (v != LSKUM_OK) return v;
        total += clouds[b].n_points;
        total_nnz += clouds[b].nbr_off[clouds[b].n_points];
    }
    if (total > INT32_MAX / 2 || total_nnz > INT32_MAX) return fail(nullptr, LSKUM_ERR_ARG, "batch too large");
    // the disjoint union of the cases' clouds
    const int32_t n = (int32_t)total;
    std::vector<double> ux, uy, unx(n, 0.0), uny(n, 0.0);
    std::vector<uint8_t> ufl;
    std::vector<int32_t> uoff(1, 0), uidx;
    ux.reserve(n);
    uy.reserve(n);
    ufl.reserve(n);
    uidx.reserve(total_nnz);
    lskum_ctx *c = new (std::nothrow) lskum_ctx();
    if (!c) return fail(nullptr, LSKUM_ERR_OOM, "host allocation failed");
    c->n_cases = n_cases;
    c->case_off.assign(1, 0);
    const bool kinetic = opts[0].farfield == LSKUM_FARFIELD_KINETIC;
    for (int32_t b = 0; b < n_cases; b++) {
        const lskum_cloud &cl = clouds[b];
        const int32_t base = (int32_t)ux.size();
        // normals not given: from the wall polygon (and the outer polygon)
        std::vector<double> cnx, cny;
        if (!cl.nx) {
            cnx.assign(cl.n_points, 0.0);
            cny.assign(cl.n_points, 0.0);
            lskum_status ps = polygon_normals(&cl, b, LSKUM_WALL, cnx.data(), cny.data());
            if (ps == LSKUM_OK && kinetic) ps = polygon_normals(&cl, b, LSKUM_OUTER, cnx.data(), cny.data());
            if (ps != LSKUM_OK) {
                delete c;
                return ps;
            }
        }
        const double *cnxp = cl.nx ? cl.nx : cnx.data(), *cnyp = cl.ny ? cl.ny : cny.data();
        for (int32_t p = 0; p < cl.n_points; p++) {
            ux.push_back(cl.x[p]);
            uy.push_back(cl.y[p]);
            ufl.push_back(cl.flag[p]);
            if (cl.flag[p] == LSKUM_WALL || (kinetic && cl.flag[p] == LSKUM_OUTER)) {
                unx[base + p] = cnxp[p];
                uny[base + p] = cnyp[p];
            }
            for (int32_t e = cl.nbr_off[p]; e < cl.nbr_off[p + 1]; e++) uidx.push_back(base + cl.nbr_idx[e]);
            uoff.push_back((int32_t)uidx.size());
            c->case_of_caller.push_back(b);
        }
        c->case_off.push_back((int32_t)ux.size());
        c->case_mach.push_back(opts[b].mach);
        c->case_aoa.push_back(opts[b].aoa_deg);
    }
    const lskum_cloud u = {n, ux.data(), uy.data(), ufl.data(), unx.data(), uny.data(), uoff.data(), uidx.data()};
    c->n = n;
    c->opts = opts[0];
    c->user_stream = (cudaStream_t)cuda_stream;
    HostPrep hp;
    lskum_status s = prepare_host(c, &u, hp);  // no CUDA call before this returns
    if (host_only) {
        if (s == LSKUM_OK) s = verify_layout(c, &u, hp);
        if (s == LSKUM_OK) {
            if (n_colours) *n_colours = c->n_colours;
            if (n_levels) *n_levels = c->n_levels;
        } else {
            g_create_error = c->err;
        }
        lskum_destroy(c);
        return s;
    }
    if (s == LSKUM_OK) {
        cudaError_t e = cudaGetDevice(&c->device);
        s = e == cudaSuccess ? upload(c, hp) : cuda_fail(c, e, "cudaGetDevice");
    }
    if (s != LSKUM_OK) {
        g_create_error = c->err;
        lskum_destroy(c);
        return s;
    }
    *out = c;
    return LSKUM_OK;
}

lskum_status lskum_validate(const lskum_cloud *clouds, const lskum_opts *opts, int32_t n_cases, int32_t *n_colours,
                            int32_t *n_levels)
{
    lskum_ctx *dummy = nullptr;
    return create_impl(clouds, opts, n_cases, nullptr, &dummy, true, n_colours, n_levels);
}

lskum_status lskum_create(const lskum_cloud *cl, const lskum_opts *opts, void *cuda_stream, lskum_ctx **out)
{
    if (!cl || !opts) {
        if (out) *out = nullptr;
        return fail(nullptr, LSKUM_ERR_ARG, "cloud or opts is NULL");
    }
    return create_impl(cl, opts, 1, cuda_stream, out);
}

lskum_status lskum_batch_create(const lskum_cloud *clouds, const lskum_opts *opts, int32_t n_cases,
                                void *cuda_stream, lskum_ctx **out)
{
    return create_impl(clouds, opts, n_cases, cuda_stream, out);
}

static lskum_status prepare_host(lskum_ctx *c, const lskum_cloud *cl, HostPrep &hp)
{
    const int32_t n = c->n;
    const int32_t *off = cl->nbr_off, *idx = cl->nbr_idx;
    c->x.assign(cl->x, cl->x + n);
    c->y.assign(cl->y, cl->y + n);
    c->flag.assign(cl->flag, cl->flag + n);
    c->nx.assign(n, 0.0);
    c->ny.assign(n, 0.0);
    const bool kinetic = c->opts.farfield == LSKUM_FARFIELD_KINETIC;
    for (int32_t p = 0; p < n; p++)
        if (c->flag[p] == LSKUM_WALL || (kinetic && c->flag[p] == LSKUM_OUTER)) {
            c->nx[p] = cl->nx[p];
            c->ny[p] = cl->ny[p];
        }

    // ---- per-slot geometry and LS weights (caller order) ----
    const int64_t nnz = off[n];
    std::vector<double> sdx(nnz), sdy(nnz), sw1(nnz, 0.0), sw2(nnz, 0.0), swgx(nnz), swgy(nnz);
    std::vector<uint8_t> &smb = hp.smb_caller;
    smb.assign(nnz, 0);
    std::vector<double> geo((size_t)G_NFIELDS * n, 0.0);
    for (int32_t p = 0; p < n; p++) {
        // frames: (t, n) at wall points (n into the fluid) and at outer points
        // of the kinetic far field (n out of the domain; their n- side is the
        // free-stream ghosts, sub-stencil 3 with LS_3(1) = -LS_2(1))
        const bool wall = c->flag[p] == LSKUM_WALL;
        const bool kouter = kinetic && c->flag[p] == LSKUM_OUTER;
        double e1x = 1.0, e1y = 0.0, e2x = 0.0, e2y = 1.0;
        if (wall || kouter) {
            e1x = c->ny[p];
            e1y = -c->nx[p];
            e2x = c->nx[p];
            e2y = c->ny[p];
        }
        geo[G_E1X * n + p] = e1x;
        geo[G_E1Y * n + p] = e1y;
        geo[G_E2X * n + p] = e2x;
        geo[G_E2Y * n + p] = e2y;
        double sdd[4] = {0, 0, 0, 0}, spp[4] = {0, 0, 0, 0}, sdp[4] = {0, 0, 0, 0};
        double s1d[4] = {0, 0, 0, 0}, s1p[4] = {0, 0, 0, 0};
        int cnt[4] = {0, 0, 0, 0};
        double sxx = 0, syy = 0, sxy = 0, dmin = INFINITY;
        for (int32_t e = off[p]; e < off[p + 1]; e++) {
            const int32_t i = idx[e];
            const double dx = c->x[i] - c->x[p], dy = c->y[i] - c->y[p];
            sdx[e] = dx;
            sdy[e] = dy;
            sxx += dx * dx;
            syy += dy * dy;
            sxy += dx * dy;
            dmin = std::min(dmin, std::sqrt(dx * dx + dy * dy));
            const double a = dx * e1x + dy * e1y, b = dx * e2x + dy * e2y;
            uint8_t mb = 0;
            if (a < 0.0) mb |= 1;
            else if (a > 0.0) mb |= 2;
            if (b < 0.0) { if (!wall) mb |= 4; }
            else if (b > 0.0) { if (!kouter) mb |= 8; }
            smb[e] = mb;
            for (int s = 0; s < 4; s++) {
                if (!(mb & (1 << s))) continue;
                const double d = s < 2 ? a : b, dp = s < 2 ? b : a;
                sdd[s] += d * d;
                spp[s] += dp * dp;
                sdp[s] += d * dp;
                s1d[s] += d;
                s1p[s] += dp;
                cnt[s]++;
            }
        }
        const int32_t deg = off[p + 1] - off[p];
        const double gdet = sxx * syy - sxy * sxy;
        if (deg < 2 || !(gdet > 1e-12 * sxx * syy))
            return fail(c, LSKUM_ERR_STENCIL, "degenerate least-squares stencil at point %d", p);
        for (int32_t e = off[p]; e < off[p + 1]; e++) {
            swgx[e] = (syy * sdx[e] - sxy * sdy[e]) / gdet;
            swgy[e] = (sxx * sdy[e] - sxy * sdx[e]) / gdet;
            geo[G_SXX * n + p] += swgx[e] * sdx[e];
            geo[G_SXY * n + p] += swgx[e] * sdy[e];
            geo[G_SYX * n + p] += swgy[e] * sdx[e];
            geo[G_SYY * n + p] += swgy[e] * sdy[e];
        }
        geo[G_DMIN * n + p] = dmin;
        if (!swept(c, p)) continue;
        double det[4];
        for (int s = 0; s < 4; s++) {
            if ((wall && s == 2) || (kouter && s == 3)) continue;
            det[s] = sdd[s] * spp[s] - sdp[s] * sdp[s];
            if (cnt[s] < 2 || !(det[s] > 1e-12 * sdd[s] * spp[s]))
                return fail(c, LSKUM_ERR_STENCIL, "degenerate split sub-stencil %d at point %d", s, p);
            geo[(G_LS1_0 + s) * n + p] = (spp[s] * s1d[s] - sdp[s] * s1p[s]) / det[s];
        }
        for (int32_t e = off[p]; e < off[p + 1]; e++) {
            const double a = sdx[e] * e1x + sdy[e] * e1y, b = sdx[e] * e2x + sdy[e] * e2y;
            for (int s = 0; s < 4; s++) {
                if (!(smb[e] & (1 << s))) continue;
                const double d = s < 2 ? a : b, dp = s < 2 ? b : a;
                const double w = (spp[s] * d - sdp[s] * dp) / det[s];
                if (s < 2) sw1[e] = w;
                else sw2[e] = w;
                geo[(G_ABS_0 + s) * n + p] += std::fabs(w);
            }
        }
        if (kouter) {  // the mirrored free-stream ghosts
            geo[G_LS1_3 * n + p] = -geo[G_LS1_2 * n + p];
            geo[G_ABS_3 * n + p] = geo[G_ABS_2 * n + p];
        }
    }

    // ---- colouring and orders ----
    c->n_colours = colour_points(n, off, idx, c->colour);
    const int32_t nc = c->n_colours;
    // sweep order (caller indices): colour by colour (Alg. 6), or wall points
    // colour by colour, then interior, then outer points (Alg. 4); ties by
    // caller index.  `skey` is the level a point belongs to; a neighbour is
    // "lower" when its key is smaller.  The serial order of Alg. 2 (wall,
    // interior, outer points, each in caller order) has no colours: its
    // levels are those of its dependency graph, a point's level one more
    // than the highest level of its earlier neighbours in the symmetrised
    // graph, so that coupled points never share a level, every earlier
    // neighbour lies in a lower level and every later one in a higher level,
    // and the level-parallel sweeps reproduce the sequential ones exactly.
    auto trank = [&](int32_t p) { return c->flag[p] == LSKUM_WALL ? 0 : (c->flag[p] == LSKUM_INTERIOR ? 1 : 2); };
    const bool wall_first = c->opts.ordering == LSKUM_ORDER_WALL_FIRST;
    const bool serial = c->opts.ordering == LSKUM_ORDER_SERIAL;
    std::vector<int64_t> depth;
    c->canon_order.resize(n);
    std::iota(c->canon_order.begin(), c->canon_order.end(), 0);
    if (serial) {
        std::stable_sort(c->canon_order.begin(), c->canon_order.end(),
                         [&](int32_t a, int32_t b) { return trank(a) < trank(b); });
        std::vector<int32_t> rank(n), rcnt, rev;
        for (int32_t k = 0; k < n; k++) rank[c->canon_order[k]] = k;
        reverse_lists(n, off, idx, rcnt, rev);
        depth.assign(n, 0);
        for (int32_t k = 0; k < n; k++) {
            const int32_t p = c->canon_order[k];
            if (!swept(c, p)) continue;
            int64_t dmax = 0;
            auto see = [&](int32_t q) {
                if (swept(c, q) && rank[q] < k) dmax = std::max(dmax, depth[q] + 1);
            };
            for (int32_t e = off[p]; e < off[p + 1]; e++) see(idx[e]);
            for (int32_t f = rcnt[p]; f < rcnt[p + 1]; f++) see(rev[f]);
            depth[p] = dmax;
        }
    }
    auto skey = [&](int32_t p) -> int64_t {
        if (serial) return depth[p];
        return wall_first ? (int64_t)trank(p) * (nc + 1) + c->colour[p] : (int64_t)c->colour[p];
    };
    if (!serial)
        std::stable_sort(c->canon_order.begin(), c->canon_order.end(),
                         [&](int32_t a, int32_t b) { return skey(a) < skey(b); });
    // internal order: level, then wall < interior < outer, then caller index
    c->perm.resize(n);
    std::iota(c->perm.begin(), c->perm.end(), 0);
    std::stable_sort(c->perm.begin(), c->perm.end(), [&](int32_t a, int32_t b) {
        if (skey(a) != skey(b)) return skey(a) < skey(b);
        return trank(a) < trank(b);
    });
    c->inv.resize(n);
    for (int32_t k = 0; k < n; k++) c->inv[c->perm[k]] = k;
    // levels: runs of equal key holding swept points; frozen outer points
    // close their level's range (or, wall-first, the last level)
    c->lvl_beg.clear();
    c->lvl_act_end.clear();
    c->lvl_end.clear();
    {
        int32_t k = 0;
        while (k < n) {
            const int64_t key = skey(c->perm[k]);
            const int32_t b = k;
            while (k < n && skey(c->perm[k]) == key && swept(c, c->perm[k])) k++;
            const int32_t ae = k;
            while (k < n && skey(c->perm[k]) == key) k++;
            if (ae > b) {
                c->lvl_beg.push_back(b);
                c->lvl_act_end.push_back(ae);
                c->lvl_end.push_back(k);
            } else if (!c->lvl_end.empty()) {
                c->lvl_end.back() = k;  // an all-outer run
            }
        }
    }
    c->n_levels = (int32_t)c->lvl_beg.size();

    // ---- sliced ELL in internal order ----
    const int32_t ld = (n + 31) / 32 * 32;
    c->ld = ld;
    const int32_t nsl = ld / 32;
    std::vector<int32_t> &slice_off = hp.slice_off, &deg = hp.deg;
    slice_off.assign(nsl + 1, 0);
    deg.assign(n, 0);
    for (int32_t s = 0; s < nsl; s++) {
        int32_t w = 0;
        for (int32_t l = 0; l < 32; l++) {
            const int32_t k = s * 32 + l;
            if (k < n) {
                const int32_t p = c->perm[k];
                w = std::max(w, off[p + 1] - off[p]);
            }
        }
        slice_off[s + 1] = slice_off[s] + 32 * w;
    }
    const int64_t ell = slice_off[nsl];
    const size_t esz = std::max<int64_t>(ell, 1);
    std::vector<int32_t> &enb = hp.enb;
    std::vector<uint8_t> &emb = hp.emb;
    std::vector<double> &edx = hp.edx, &edy = hp.edy, &ew1 = hp.ew1, &ew2 = hp.ew2, &egx = hp.egx, &egy = hp.egy;
    enb.assign(esz, 0);
    emb.assign(esz, 0);
    for (auto *v : {&edx, &edy, &ew1, &ew2, &egx, &egy, &hp.exx, &hp.exy, &hp.eyx, &hp.eyy}) v->assign(esz, 0.0);
    for (int32_t k = 0; k < n; k++) {
        const int32_t p = c->perm[k];
        deg[k] = off[p + 1] - off[p];
        const int64_t base = slice_off[k / 32] + (k % 32);
        const int32_t w = (slice_off[k / 32 + 1] - slice_off[k / 32]) / 32;
        for (int32_t j = 0; j < w; j++) enb[base + 32 * j] = k;  // padding: self, never read
        for (int32_t j = 0; j < deg[k]; j++) {
            const int64_t e = off[p] + j, t = base + 32 * j;
            enb[t] = c->inv[idx[e]];
            emb[t] = smb[e];
            edx[t] = 0.5 * sdx[e];  // half offsets (exact): the residual's reconstruction
            edy[t] = 0.5 * sdy[e];  // steps q - (dx, dy)/2 . grad q
            ew1[t] = sw1[e];
            ew2[t] = sw2[e];
            egx[t] = swgx[e];
            egy[t] = swgy[e];
            hp.exx[t] = swgx[e] * sdx[e];
            hp.exy[t] = swgx[e] * sdy[e];
            hp.eyx[t] = swgy[e] * sdx[e];
            hp.eyy[t] = swgy[e] * sdy[e];
        }
    }
    // LU-SGS lists: for each point its slots whose neighbour is earlier (lower)
    // or later (upper) in the sweep order; frozen neighbours (increment 0)
    // and slots in no split sub-stencil contribute nothing and are left out
    hp.lo_off.assign(n + 1, 0);
    hp.up_off.assign(n + 1, 0);
    for (int32_t k = 0; k < n; k++) {
        const int32_t p = c->perm[k];
        if (swept(c, p)) {
            for (int32_t e = off[p]; e < off[p + 1]; e++) {
                const int32_t q = idx[e];
                if (!swept(c, q) || smb[e] == 0) continue;
                const bool lower = skey(q) < skey(p);
                (lower ? hp.lo_nbr : hp.up_nbr).push_back(c->inv[q]);
                (lower ? hp.lo_mb : hp.up_mb).push_back(smb[e]);
                (lower ? hp.lo_w1 : hp.up_w1).push_back(sw1[e]);
                (lower ? hp.lo_w2 : hp.up_w2).push_back(sw2[e]);
            }
        }
        hp.lo_off[k + 1] = (int32_t)hp.lo_nbr.size();
        hp.up_off[k + 1] = (int32_t)hp.up_nbr.size();
    }
    // per level, points by decreasing list length (a warp's groups then share a trip count)
    hp.sw_fwd.assign(std::max(n, 1), 0);
    hp.sw_bwd.assign(std::max(n, 1), 0);
    for (int32_t l = 0; l < c->n_levels; l++) {
        const int32_t b = c->lvl_beg[l], e = c->lvl_act_end[l];
        for (int32_t k = b; k < e; k++) hp.sw_fwd[k] = hp.sw_bwd[k] = k;
        auto lo_len = [&](int32_t k) { return hp.lo_off[k + 1] - hp.lo_off[k]; };
        auto up_len = [&](int32_t k) { return hp.up_off[k + 1] - hp.up_off[k]; };
        std::stable_sort(hp.sw_fwd.begin() + b, hp.sw_fwd.begin() + e,
                         [&](int32_t a, int32_t z) { return lo_len(a) > lo_len(z); });
        std::stable_sort(hp.sw_bwd.begin() + b, hp.sw_bwd.begin() + e,
                         [&](int32_t a, int32_t z) { return up_len(a) > up_len(z); });
    }
    // packed sweep form, per level:
    // - points in a (t, n) frame (wall points, and outer points under the
    //   kinetic far field), which form their Jacobian products per slot: their
    //   slots packed into warps of 32 lanes by best fit (longest lists first; a
    //   point with an empty list takes one slot with membership 0), a point
    //   never straddling two warps;
    // - interior points, which gather their neighbours' stored axis products:
    //   kLanesPerPoint lanes per point, in groups of kPointsPerWarp points in
    //   sweep order (decreasing list length), each group's lists in ELL
    //   layout (slot j of point p at lp_goff[g] + 32 (j / L) + L p + j % L,
    //   L = kLanesPerPoint).
    c->pk_ok = true;
    for (int32_t k = 0; k < n; k++)
        if (hp.lo_off[k + 1] - hp.lo_off[k] > 32 || hp.up_off[k + 1] - hp.up_off[k] > 32) c->pk_ok = false;
    for (int dir = 0; dir < 2 && c->pk_ok; dir++) {
        const std::vector<int32_t> &so = dir == 0 ? hp.sw_fwd : hp.sw_bwd;
        const std::vector<int32_t> &loff = dir == 0 ? hp.lo_off : hp.up_off;
        const std::vector<int32_t> &lnbr = dir == 0 ? hp.lo_nbr : hp.up_nbr;
        const std::vector<uint8_t> &lmb = dir == 0 ? hp.lo_mb : hp.up_mb;
        const std::vector<double> &lw1 = dir == 0 ? hp.lo_w1 : hp.up_w1, &lw2 = dir == 0 ? hp.lo_w2 : hp.up_w2;
        std::vector<int32_t> &lw = c->pk_lw[dir], &lg = c->lp_lg[dir];
        lw.assign(1, 0);
        lg.assign(1, 0);
        hp.lp_goff[dir].assign(1, 0);
        int32_t nw = 0, ng = 0;
        for (int32_t l = 0; l < c->n_levels; l++) {
            // framed points: best fit, warps by free lanes (bucket r holds warps with r free)
            std::vector<std::vector<int32_t>> members;  // positions per warp of this level
            std::vector<int32_t> inner;                 // interior points (internal index), sweep order
            std::vector<std::vector<int32_t>> bucket(33);
            for (int32_t pos = c->lvl_beg[l]; pos < c->lvl_act_end[l]; pos++) {
                const int32_t k = so[pos];
                if (c->flag[c->perm[k]] == LSKUM_INTERIOR) {
                    inner.push_back(k);
                    continue;
                }
                const int32_t len = std::max(1, loff[k + 1] - loff[k]);
                int32_t w = -1;
                for (int32_t r = len; r <= 32 && w < 0; r++)
                    if (!bucket[r].empty()) {
                        w = bucket[r].back();
                        bucket[r].pop_back();
                        bucket[r - len].push_back(w);
                    }
                if (w < 0) {
                    w = (int32_t)members.size();
                    members.emplace_back();
                    bucket[32 - len].push_back(w);
                }
                members[w].push_back(pos);
            }
            for (const auto &mw : members) {
                int32_t lane = 0, longest = 1;
                for (int32_t pos : mw) longest = std::max(longest, loff[so[pos] + 1] - loff[so[pos]]);
                uint8_t steps = 0;
                while ((1 << steps) < longest) steps++;
                hp.pk_steps[dir].push_back(steps);
                for (int32_t pos : mw) {
                    const int32_t k = so[pos];
                    const int32_t b = loff[k], e = loff[k + 1];
                    if (e == b) {
                        hp.pk_pt[dir].push_back(pos);
                        hp.pk_nbr[dir].push_back(k);
                        hp.pk_mb[dir].push_back(0);
                        hp.pk_w1[dir].push_back(0.0);
                        hp.pk_w2[dir].push_back(0.0);
                        lane++;
                    }
                    for (int32_t j = b; j < e; j++, lane++) {
                        hp.pk_pt[dir].push_back(pos);
                        hp.pk_nbr[dir].push_back(lnbr[j]);
                        hp.pk_mb[dir].push_back(lmb[j]);
                        hp.pk_w1[dir].push_back(lw1[j]);
                        hp.pk_w2[dir].push_back(lw2[j]);
                    }
                }
                for (; lane < 32; lane++) {  // padding
                    hp.pk_pt[dir].push_back(-1);
                    hp.pk_nbr[dir].push_back(0);
                    hp.pk_mb[dir].push_back(0);
                    hp.pk_w1[dir].push_back(0.0);
                    hp.pk_w2[dir].push_back(0.0);
                }
            }
            nw += (int32_t)members.size();
            lw.push_back(nw);
            // interior points: groups of kPointsPerWarp points, ELL lists
            constexpr int L = kLanesPerPoint;
            for (size_t g0 = 0; g0 < inner.size(); g0 += kPointsPerWarp) {
                int32_t width = 0;  // rows of 32 slots
                for (size_t t = 0; t < (size_t)kPointsPerWarp; t++) {
                    const int32_t k = g0 + t < inner.size() ? inner[g0 + t] : -1;
                    const int32_t len = k >= 0 ? loff[k + 1] - loff[k] : 0;
                    hp.lp_k[dir].push_back(k);
                    hp.lp_len[dir].push_back(len);
                    width = std::max(width, (len + L - 1) / L);
                }
                const int32_t base = hp.lp_goff[dir].back();
                hp.lp_goff[dir].push_back(base + 32 * width);
                hp.lp_nbr[dir].resize((size_t)base + 32 * width, 0);
                hp.lp_mb[dir].resize((size_t)base + 32 * width, 0);
                hp.lp_w1[dir].resize((size_t)base + 32 * width, 0.0);
                hp.lp_w2[dir].resize((size_t)base + 32 * width, 0.0);
                for (size_t t = 0; t < (size_t)kPointsPerWarp && g0 + t < inner.size(); t++) {
                    const int32_t k = inner[g0 + t];
                    for (int32_t j = 0; j < loff[k + 1] - loff[k]; j++) {
                        const size_t e = (size_t)base + 32 * (size_t)(j / L) + L * t + j % L;
                        hp.lp_nbr[dir][e] = lnbr[loff[k] + j];
                        hp.lp_mb[dir][e] = lmb[loff[k] + j];
                        hp.lp_w1[dir][e] = lw1[loff[k] + j];
                        hp.lp_w2[dir][e] = lw2[loff[k] + j];
                    }
                }
                ng++;
            }
            lg.push_back(ng);
        }
    }
    for (auto *v : {&hp.lo_nbr, &hp.up_nbr}) if (v->empty()) v->push_back(0);
    for (auto *v : {&hp.lo_mb, &hp.up_mb}) if (v->empty()) v->push_back(0);
    for (auto *v : {&hp.lo_w1, &hp.lo_w2, &hp.up_w1, &hp.up_w2}) if (v->empty()) v->push_back(0.0);

    std::vector<double> &geo_i = hp.geo_i, &wnx = hp.wnx, &wny = hp.wny;
    std::vector<uint8_t> &fl_i = hp.fl_i;
    geo_i.assign((size_t)G_NFIELDS * ld, 0.0);
    wnx.assign(ld, 0.0);
    wny.assign(ld, 0.0);
    fl_i.assign(ld, LSKUM_OUTER);
    for (int32_t k = 0; k < n; k++) {
        const int32_t p = c->perm[k];
        for (int f = 0; f < G_NFIELDS; f++) geo_i[(size_t)f * ld + k] = geo[(size_t)f * n + p];
        wnx[k] = c->nx[p];
        wny[k] = c->ny[p];
        fl_i[k] = c->flag[p];
    }

    // per-case norm blocks over caller positions (never straddling two cases)
    hp.case_blk.assign(1, 0);
    hp.blk_pos.clear();
    hp.blk_case.clear();
    for (int32_t b = 0; b < c->n_cases; b++) {
        for (int32_t p0 = c->case_off[b]; p0 < c->case_off[b + 1]; p0 += 256) {
            hp.blk_pos.push_back(p0);
            hp.blk_case.push_back(b);
        }
        hp.case_blk.push_back((int32_t)hp.blk_pos.size());
    }
    hp.blk_pos.push_back(n);  // block j ends where block j + 1 (or the next case) starts
    hp.case_of_i.assign(ld, 0);
    for (int32_t k = 0; k < n; k++) hp.case_of_i[k] = c->case_of_caller[c->perm[k]];
    return LSKUM_OK;
}

static lskum_status upload(lskum_ctx *c, HostPrep &hp)
{
    const int32_t n = c->n, ld = c->ld, nsl = ld / 32;
    std::vector<int32_t> &slice_off = hp.slice_off, &deg = hp.deg, &enb = hp.enb;
    std::vector<uint8_t> &emb = hp.emb, &fl_i = hp.fl_i;
    std::vector<double> &edx = hp.edx, &edy = hp.edy, &ew1 = hp.ew1, &ew2 = hp.ew2, &egx = hp.egx, &egy = hp.egy;
    std::vector<double> &geo_i = hp.geo_i, &wnx = hp.wnx, &wny = hp.wny;
    // ---- device memory ----
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamCreate");
    e = cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
    e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(c, e, "side stream");
    Arena &A = c->arena;
    Dev &d = c->dev;
    d.n = n;
    d.ld = ld;
    d.n_slices = nsl;
    uint8_t *dfl = A.alloc<uint8_t>(ld);
    double *dwnx = A.alloc<double>(ld), *dwny = A.alloc<double>(ld);
    double *dgeo = A.alloc<double>((size_t)G_NFIELDS * ld);
    int32_t *dso = A.alloc<int32_t>(nsl + 1), *ddeg = A.alloc<int32_t>(n), *dnb = A.alloc<int32_t>(enb.size());
    uint8_t *dmb = A.alloc<uint8_t>(emb.size());
    double *ddx = A.alloc<double>(edx.size()), *ddy = A.alloc<double>(edx.size());
    double *dw1 = A.alloc<double>(edx.size()), *dw2 = A.alloc<double>(edx.size());
    double *dgx = A.alloc<double>(edx.size()), *dgy = A.alloc<double>(edx.size());
    double *dxx = A.alloc<double>(edx.size()), *dxy = A.alloc<double>(edx.size());
    double *dyx = A.alloc<double>(edx.size()), *dyy = A.alloc<double>(edx.size());
    for (int s = 0; s < 2; s++) {
        d.set[s].U = A.alloc<double>(4 * (size_t)ld);
        d.set[s].q = A.alloc<double>(4 * (size_t)ld);
        d.set[s].prim = A.alloc<double>((size_t)kPrimStride * ld);
        d.gq[s] = A.alloc<double>(8 * (size_t)ld);
    }
    int32_t *dlo_off = A.alloc<int32_t>(n + 1), *dup_off = A.alloc<int32_t>(n + 1);
    int32_t *dlo_nbr = A.alloc<int32_t>(hp.lo_nbr.size()), *dup_nbr = A.alloc<int32_t>(hp.up_nbr.size());
    uint8_t *dlo_mb = A.alloc<uint8_t>(hp.lo_mb.size()), *dup_mb = A.alloc<uint8_t>(hp.up_mb.size());
    double *dlo_w1 = A.alloc<double>(hp.lo_w1.size()), *dlo_w2 = A.alloc<double>(hp.lo_w2.size());
    double *dup_w1 = A.alloc<double>(hp.up_w1.size()), *dup_w2 = A.alloc<double>(hp.up_w2.size());
    int32_t *dsw_fwd = A.alloc<int32_t>(hp.sw_fwd.size()), *dsw_bwd = A.alloc<int32_t>(hp.sw_bwd.size());
    // mixed precision: FP32 increments, primal records and weights
    const bool mixed = c->opts.precision == 1;
    std::vector<float> flo_w1, flo_w2, fup_w1, fup_w2;
    float *dlo_w1f = nullptr, *dlo_w2f = nullptr, *dup_w1f = nullptr, *dup_w2f = nullptr;
    d.dUsf = d.dUf = nullptr;
    for (int s = 0; s < 2; s++) d.set[s].primf = nullptr;
    if (mixed) {
        for (auto pr : {std::make_pair(&hp.lo_w1, &flo_w1), std::make_pair(&hp.lo_w2, &flo_w2),
                        std::make_pair(&hp.up_w1, &fup_w1), std::make_pair(&hp.up_w2, &fup_w2)})
            pr.second->assign(pr.first->begin(), pr.first->end());
        dlo_w1f = A.alloc<float>(flo_w1.size());
        dlo_w2f = A.alloc<float>(flo_w2.size());
        dup_w1f = A.alloc<float>(fup_w1.size());
        dup_w2f = A.alloc<float>(fup_w2.size());
        d.dUsf = A.alloc<float>(4 * (size_t)ld);
        d.dUf = A.alloc<float>(4 * (size_t)ld);
        for (int s = 0; s < 2; s++) d.set[s].primf = A.alloc<float>((size_t)kPrimStride * ld);
    }
    // packed sweep form (arrays of at least one element, so that a level set
    // without framed points, or without interior points, still has them)
    std::vector<float> pkf[2][2], lpf[2][2];
    for (int dir = 0; dir < 2; dir++) {
        d.pk_pt[dir] = d.pk_nbr[dir] = nullptr;
        d.pk_mb[dir] = d.pk_steps[dir] = nullptr;
        d.pk_w1[dir] = d.pk_w2[dir] = nullptr;
        d.pk_w1f[dir] = d.pk_w2f[dir] = nullptr;
        d.lp_k[dir] = d.lp_len[dir] = d.lp_goff[dir] = d.lp_nbr[dir] = nullptr;
        d.lp_mb[dir] = nullptr;
        d.lp_w1[dir] = d.lp_w2[dir] = nullptr;
        d.lp_w1f[dir] = d.lp_w2f[dir] = nullptr;
        if (!c->pk_ok) continue;
        const size_t m = std::max<size_t>(hp.pk_pt[dir].size(), 1);
        d.pk_pt[dir] = A.alloc<int32_t>(m);
        d.pk_nbr[dir] = A.alloc<int32_t>(m);
        d.pk_mb[dir] = A.alloc<uint8_t>(m);
        d.pk_steps[dir] = A.alloc<uint8_t>(std::max<size_t>(hp.pk_steps[dir].size(), 1));
        d.pk_w1[dir] = A.alloc<double>(m);
        d.pk_w2[dir] = A.alloc<double>(m);
        const size_t nk = std::max<size_t>(hp.lp_k[dir].size(), 1), ne = std::max<size_t>(hp.lp_nbr[dir].size(), 1);
        d.lp_k[dir] = A.alloc<int32_t>(nk);
        d.lp_len[dir] = A.alloc<int32_t>(nk);
        d.lp_goff[dir] = A.alloc<int32_t>(hp.lp_goff[dir].size());
        d.lp_nbr[dir] = A.alloc<int32_t>(ne);
        d.lp_mb[dir] = A.alloc<uint8_t>(ne);
        d.lp_w1[dir] = A.alloc<double>(ne);
        d.lp_w2[dir] = A.alloc<double>(ne);
        if (mixed) {
            pkf[dir][0].assign(hp.pk_w1[dir].begin(), hp.pk_w1[dir].end());
            pkf[dir][1].assign(hp.pk_w2[dir].begin(), hp.pk_w2[dir].end());
            d.pk_w1f[dir] = A.alloc<float>(m);
            d.pk_w2f[dir] = A.alloc<float>(m);
            lpf[dir][0].assign(hp.lp_w1[dir].begin(), hp.lp_w1[dir].end());
            lpf[dir][1].assign(hp.lp_w2[dir].begin(), hp.lp_w2[dir].end());
            d.lp_w1f[dir] = A.alloc<float>(ne);
            d.lp_w2f[dir] = A.alloc<float>(ne);
        }
    }
    // per-point axis Jacobian products of the packed form (x+, x-, y+, y-)
    d.jc = nullptr;
    d.jcf = nullptr;
    if (c->pk_ok) {
        if (mixed) d.jcf = A.alloc<float>(16 * (size_t)ld);
        else d.jc = A.alloc<double>(16 * (size_t)ld);
    }
    // the framed points' Jacobians of the packed form (exact products):
    // per slot lane a weighted 4x4 matrix, per framed point its four axis
    // Jacobians; framed points numbered in internal order
    std::vector<int32_t> h_fidx, h_fpt;
    for (int dir = 0; dir < 2; dir++) {
        d.pk_jm[dir] = nullptr;
        d.pk_jmf[dir] = nullptr;
        d.pk_lanes[dir] = 0;
    }
    d.fj = nullptr;
    d.fjf = nullptr;
    d.fidx = d.fpt = nullptr;
    d.nf = 0;
    if (c->pk_ok && c->opts.jvp == LSKUM_JVP_EXACT) {
        h_fidx.assign(ld, -1);
        for (int32_t k = 0; k < n; k++) {
            const uint8_t fl = c->flag[c->perm[k]];
            if (fl == LSKUM_WALL || (fl == LSKUM_OUTER && c->opts.farfield == LSKUM_FARFIELD_KINETIC)) {
                h_fidx[k] = (int32_t)h_fpt.size();
                h_fpt.push_back(k);
            }
        }
        d.nf = (int32_t)h_fpt.size();
        for (int dir = 0; dir < 2; dir++) {
            d.pk_lanes[dir] = (int32_t)hp.pk_pt[dir].size();
            const size_t m = 16 * std::max<size_t>(hp.pk_pt[dir].size(), 1);
            if (mixed) d.pk_jmf[dir] = A.alloc<float>(m);
            else d.pk_jm[dir] = A.alloc<double>(m);
        }
        const size_t mf = 64 * std::max<size_t>(h_fpt.size(), 1);
        if (mixed) d.fjf = A.alloc<float>(mf);
        else d.fj = A.alloc<double>(mf);
        d.fidx = A.alloc<int32_t>(ld);
        d.fpt = A.alloc<int32_t>(std::max<size_t>(h_fpt.size(), 1));
    }
    c->launch.pk_lw[0] = c->pk_ok ? c->pk_lw[0].data() : nullptr;
    c->launch.pk_lw[1] = c->pk_ok ? c->pk_lw[1].data() : nullptr;
    c->launch.lp_lg[0] = c->pk_ok ? c->lp_lg[0].data() : nullptr;
    c->launch.lp_lg[1] = c->pk_ok ? c->lp_lg[1].data() : nullptr;
    d.g1x = A.alloc<double>(4 * (size_t)ld);
    d.g1y = A.alloc<double>(4 * (size_t)ld);
    d.R = A.alloc<double>(4 * (size_t)ld);
    d.D = A.alloc<double>(ld);
    d.iD = A.alloc<double>(ld);
    d.dUs = A.alloc<double>(4 * (size_t)ld);
    d.dU = A.alloc<double>(4 * (size_t)ld);
    // launch shape: enough threads per point to fill the GPU on small clouds
    c->launch.res_block = 128;
    c->launch.tpp = n >= 100000 ? 1 : (n >= 50000 ? 2 : (n >= 25000 ? 4 : 8));
    c->launch.sweep_lanes = 4;
    d.n_blk = (int32_t)hp.blk_case.size();
    d.n_cases = c->n_cases;
    d.blk = A.alloc<double>(4 * (size_t)d.n_blk);
    int32_t *dblk_pos = A.alloc<int32_t>(hp.blk_pos.size()), *dblk_case = A.alloc<int32_t>(hp.blk_case.size());
    int32_t *dcase_blk = A.alloc<int32_t>(hp.case_blk.size()), *dinv = A.alloc<int32_t>(n);
    int32_t *dcase_of = A.alloc<int32_t>(ld);
    c->ctrl = A.alloc<Ctrl>(1);
    c->case_state = A.alloc<int32_t>(c->n_cases);
    c->case_it = A.alloc<int32_t>(c->n_cases);
    c->case_hist0 = A.alloc<double>(c->n_cases);
    c->case_err = A.alloc<int32_t>(c->n_cases);
    c->case_bad = A.alloc<int32_t>(c->n_cases);
    c->hist_cap = 4096;
    c->hist = A.alloc<double>((size_t)c->n_cases * c->hist_cap);
    c->hist4 = A.alloc<double>((size_t)c->n_cases * c->hist_cap * 4);
    c->dscratch = A.alloc<double>(4 * (size_t)ld);
    if (A.err != cudaSuccess) return cuda_fail(c, A.err, "cudaMalloc");
    e = cudaMemset(c->ctrl, 0, sizeof(Ctrl));
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemset");
    d.flag = dfl;
    d.wnx = dwnx;
    d.wny = dwny;
    d.geo = dgeo;
    d.slice_off = dso;
    d.deg = ddeg;
    d.nbr = dnb;
    d.memb = dmb;
    d.nhx = ddx;
    d.nhy = ddy;
    d.w1 = dw1;
    d.w2 = dw2;
    d.wgx = dgx;
    d.wgy = dgy;
    d.gxx = dxx;
    d.gxy = dxy;
    d.gyx = dyx;
    d.gyy = dyy;
    d.ctrl = c->ctrl;
    d.case_state = c->case_state;
    d.blk_pos = dblk_pos;
    d.blk_case = dblk_case;
    d.case_blk = dcase_blk;
    d.inv = dinv;
    d.case_of = dcase_of;
    d.lo_off = dlo_off;
    d.up_off = dup_off;
    d.lo_nbr = dlo_nbr;
    d.up_nbr = dup_nbr;
    d.lo_mb = dlo_mb;
    d.up_mb = dup_mb;
    d.lo_w1 = dlo_w1;
    d.lo_w2 = dlo_w2;
    d.up_w1 = dup_w1;
    d.up_w2 = dup_w2;
    d.sw_fwd = dsw_fwd;
    d.sw_bwd = dsw_bwd;
    d.lo_w1f = dlo_w1f;
    d.lo_w2f = dlo_w2f;
    d.up_w1f = dup_w1f;
    d.up_w2f = dup_w2f;
    d.precision = c->opts.precision;
    d.cfl = c->opts.cfl;
    d.ramp = c->opts.cfl_ramp_iters;
    d.K = c->opts.inner_iters;
    d.first_order = c->opts.first_order_iters;
    d.jvp = c->opts.jvp;
    d.scheme = c->opts.scheme;
    d.lusgs = c->opts.lusgs;
    d.farfield = c->opts.farfield;
    double *dcase_uinf = A.alloc<double>(4 * (size_t)c->n_cases);
    if (A.err != cudaSuccess) return cuda_fail(c, A.err, "cudaMalloc");
    d.case_uinf = dcase_uinf;
    std::vector<double> cuinf(4 * (size_t)c->n_cases);
    for (int32_t b = 0; b < c->n_cases; b++) {
        double ub, vb;
        host_free_stream(c, b, &ub, &vb);
        host_prim_to_cons(1.0, ub, vb, 1.0 / 1.4, &cuinf[4 * b]);  // as the start state below
    }
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(dfl, fl_i.data(), ld);
    up(dwnx, wnx.data(), ld * sizeof(double));
    up(dwny, wny.data(), ld * sizeof(double));
    up(dgeo, geo_i.data(), geo_i.size() * sizeof(double));
    up(dso, slice_off.data(), slice_off.size() * sizeof(int32_t));
    up(ddeg, deg.data(), n * sizeof(int32_t));
    up(dnb, enb.data(), enb.size() * sizeof(int32_t));
    up(dmb, emb.data(), emb.size());
    up(ddx, edx.data(), edx.size() * sizeof(double));
    up(ddy, edy.data(), edy.size() * sizeof(double));
    up(dw1, ew1.data(), ew1.size() * sizeof(double));
    up(dw2, ew2.data(), ew2.size() * sizeof(double));
    up(dgx, egx.data(), egx.size() * sizeof(double));
    up(dgy, egy.data(), egy.size() * sizeof(double));
    up(dxx, hp.exx.data(), hp.exx.size() * sizeof(double));
    up(dxy, hp.exy.data(), hp.exy.size() * sizeof(double));
    up(dyx, hp.eyx.data(), hp.eyx.size() * sizeof(double));
    up(dyy, hp.eyy.data(), hp.eyy.size() * sizeof(double));
    up(dlo_off, hp.lo_off.data(), hp.lo_off.size() * sizeof(int32_t));
    up(dup_off, hp.up_off.data(), hp.up_off.size() * sizeof(int32_t));
    up(dlo_nbr, hp.lo_nbr.data(), hp.lo_nbr.size() * sizeof(int32_t));
    up(dup_nbr, hp.up_nbr.data(), hp.up_nbr.size() * sizeof(int32_t));
    up(dlo_mb, hp.lo_mb.data(), hp.lo_mb.size());
    up(dup_mb, hp.up_mb.data(), hp.up_mb.size());
    up(dlo_w1, hp.lo_w1.data(), hp.lo_w1.size() * sizeof(double));
    up(dlo_w2, hp.lo_w2.data(), hp.lo_w2.size() * sizeof(double));
    up(dup_w1, hp.up_w1.data(), hp.up_w1.size() * sizeof(double));
    up(dup_w2, hp.up_w2.data(), hp.up_w2.size() * sizeof(double));
    up(dsw_fwd, hp.sw_fwd.data(), hp.sw_fwd.size() * sizeof(int32_t));
    up(dsw_bwd, hp.sw_bwd.data(), hp.sw_bwd.size() * sizeof(int32_t));
    up(dblk_pos, hp.blk_pos.data(), hp.blk_pos.size() * sizeof(int32_t));
    up(dblk_case, hp.blk_case.data(), hp.blk_case.size() * sizeof(int32_t));
    up(dcase_blk, hp.case_blk.data(), hp.case_blk.size() * sizeof(int32_t));
    up(dinv, c->inv.data(), n * sizeof(int32_t));
    up(dcase_of, hp.case_of_i.data(), ld * sizeof(int32_t));
    up(dcase_uinf, cuinf.data(), cuinf.size() * sizeof(double));
    for (int dir = 0; dir < 2; dir++) {
        if (!d.pk_pt[dir]) continue;
        const size_t m = hp.pk_pt[dir].size(), nk = hp.lp_k[dir].size(), ne = hp.lp_nbr[dir].size();
        up((void *)d.pk_pt[dir], hp.pk_pt[dir].data(), m * sizeof(int32_t));
        up((void *)d.pk_nbr[dir], hp.pk_nbr[dir].data(), m * sizeof(int32_t));
        up((void *)d.pk_mb[dir], hp.pk_mb[dir].data(), m);
        up((void *)d.pk_steps[dir], hp.pk_steps[dir].data(), hp.pk_steps[dir].size());
        up((void *)d.pk_w1[dir], hp.pk_w1[dir].data(), m * sizeof(double));
        up((void *)d.pk_w2[dir], hp.pk_w2[dir].data(), m * sizeof(double));
        up((void *)d.lp_k[dir], hp.lp_k[dir].data(), nk * sizeof(int32_t));
        up((void *)d.lp_len[dir], hp.lp_len[dir].data(), nk * sizeof(int32_t));
        up((void *)d.lp_goff[dir], hp.lp_goff[dir].data(), hp.lp_goff[dir].size() * sizeof(int32_t));
        up((void *)d.lp_nbr[dir], hp.lp_nbr[dir].data(), ne * sizeof(int32_t));
        up((void *)d.lp_mb[dir], hp.lp_mb[dir].data(), ne);
        up((void *)d.lp_w1[dir], hp.lp_w1[dir].data(), ne * sizeof(double));
        up((void *)d.lp_w2[dir], hp.lp_w2[dir].data(), ne * sizeof(double));
        if (d.pk_w1f[dir]) {
            up((void *)d.pk_w1f[dir], pkf[dir][0].data(), m * sizeof(float));
            up((void *)d.pk_w2f[dir], pkf[dir][1].data(), m * sizeof(float));
            up((void *)d.lp_w1f[dir], lpf[dir][0].data(), ne * sizeof(float));
            up((void *)d.lp_w2f[dir], lpf[dir][1].data(), ne * sizeof(float));
        }
    }
    if (d.fidx) {
        up((void *)d.fidx, h_fidx.data(), ld * sizeof(int32_t));
        up((void *)d.fpt, h_fpt.data(), h_fpt.size() * sizeof(int32_t));
    }
    if (e == cudaSuccess && d.jc) e = cudaMemset(d.jc, 0, 16 * (size_t)ld * sizeof(double));
    if (e == cudaSuccess && d.jcf) e = cudaMemset(d.jcf, 0, 16 * (size_t)ld * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->case_state, 0, c->n_cases * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->case_it, 0, c->n_cases * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->case_hist0, 0, c->n_cases * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(c->case_err, 0, c->n_cases * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->case_bad, 0x7f, c->n_cases * sizeof(int32_t));
    if (mixed) {
        up(dlo_w1f, flo_w1.data(), flo_w1.size() * sizeof(float));
        up(dlo_w2f, flo_w2.data(), flo_w2.size() * sizeof(float));
        up(dup_w1f, fup_w1.data(), fup_w1.size() * sizeof(float));
        up(dup_w2f, fup_w2.data(), fup_w2.size() * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(d.dUsf, 0, 4 * (size_t)ld * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(d.dUf, 0, 4 * (size_t)ld * sizeof(float));
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
    // zero intermediates; D = 1 at outer points (never written by the kernels)
    for (double *p : {d.R, d.dUs, d.dU, d.gq[0], d.gq[0] + 4 * (size_t)ld, d.gq[1], d.gq[1] + 4 * (size_t)ld})
        if (e == cudaSuccess) e = cudaMemset(p, 0, 4 * (size_t)ld * sizeof(double));
    std::vector<double> ones(ld, 1.0);
    up(d.D, ones.data(), ld * sizeof(double));
    up(d.iD, ones.data(), ld * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemset");

    // host arrays may go straight to and from the reorder kernels where the
    // device reads and writes pageable host memory (off by default: not
    // faster on GB300, see lskum_set_host_io)
    int pageable = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, c->device) != cudaSuccess) pageable = 0;
    c->host_direct_ok = pageable == 1;
    c->host_direct = false;

    // the function tables the sweeps read from global memory
    e = launch_init_math(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "initialising the function tables");

    // ---- free-stream start ----
    std::vector<double> rho(n, 1.0), uu(n), vv(n), pp(n, 1.0 / 1.4);
    for (int32_t b = 0; b < c->n_cases; b++) {
        double ub, vb;
        host_free_stream(c, b, &ub, &vb);
        for (int32_t p = c->case_off[b]; p < c->case_off[b + 1]; p++) {
            uu[p] = ub;
            vv[p] = vb;
        }
    }
    lskum_status s = lskum_set_state(c, rho.data(), uu.data(), vv.data(), pp.data());
    if (s != LSKUM_OK) return s;

    return build_graphs(c);
}

// (Re)capture one CUDA graph per state parity with the current launch shape.
static lskum_status build_graphs(lskum_ctx *c)
{
    for (auto &g : c->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (int par = 0; par < 2; par++) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
        int launches = 0;
        Launch L = c->launch;  // captured: the framed Jacobians on the side branch
        L.side = c->side;
        L.fork = c->ev_fork;
        L.join = c->ev_join;
        cudaError_t le = launch_iteration(c->dev, L, par, c->n_levels, c->lvl_beg.data(),
                                          c->lvl_act_end.data(), c->lvl_end.data(), c->stream, &launches);
        e = cudaStreamEndCapture(c->stream, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(c, le, "kernel launch during capture");
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->graph[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
        c->launches_per_iter = launches;
    }
    return LSKUM_OK;
}

void lskum_destroy(lskum_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &g : c->graph)
        if (g) cudaGraphExecDestroy(g);
    c->arena.release();
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"

namespace {

// order the internal stream after the caller's stream
cudaError_t join_user(lskum_ctx *c)
{
    if (!c->user_stream) return cudaSuccess;
    cudaError_t e = cudaEventRecord(c->ev, c->user_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev, 0);
    return e;
}

cudaError_t release_user(lskum_ctx *c)
{
    if (!c->user_stream) return cudaSuccess;
    cudaError_t e = cudaEventRecord(c->ev, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->user_stream, c->ev, 0);
    return e;
}

lskum_status read_ctrl(lskum_ctx *c, Ctrl *h)
{
    cudaError_t e = cudaMemcpyAsync(h, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the control block");
    return LSKUM_OK;
}

// Write the host copy of the control block (with the context's per-case
// pointers filled in) to the device and wait for it.
lskum_status write_ctrl(lskum_ctx *c, Ctrl &h)
{
    h.n_cases = c->n_cases;
    h.case_state = c->case_state;
    h.case_it = c->case_it;
    h.case_hist0 = c->case_hist0;
    h.case_err = c->case_err;
    h.case_bad = c->case_bad;
    h.hist = c->hist;
    h.hist4 = c->hist4;
    h.hist_cap = c->hist_cap;
    cudaError_t e = cudaMemcpyAsync(c->ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "writing the control block");
    return LSKUM_OK;
}

// Per-case counters.  A new state (`fresh`) clears everything: every case
// runs again, failures are forgotten and, with `history`, the histories are
// cleared.  Otherwise stopped cases run again and failed cases stay failed.
lskum_status reset_cases(lskum_ctx *c, bool history, bool fresh)
{
    cudaError_t e = cudaSuccess;
    if (fresh) {
        e = cudaMemsetAsync(c->case_state, 0, c->n_cases * sizeof(int32_t), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->case_err, 0, c->n_cases * sizeof(int32_t), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->case_bad, 0x7f, c->n_cases * sizeof(int32_t), c->stream);
    } else {
        std::vector<int32_t> st(c->n_cases);
        e = cudaMemcpyAsync(st.data(), c->case_state, c->n_cases * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        for (auto &x : st) x = (x == kFailed || x == kFailedNow) ? (int32_t)kFailed : (int32_t)kRunning;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->case_state, st.data(), c->n_cases * sizeof(int32_t), cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (history && e == cudaSuccess) e = cudaMemsetAsync(c->case_it, 0, c->n_cases * sizeof(int32_t), c->stream);
    if (history && e == cudaSuccess) e = cudaMemsetAsync(c->case_hist0, 0, c->n_cases * sizeof(double), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "resetting the cases");
    return LSKUM_OK;
}

lskum_status read_case_arrays(lskum_ctx *c, std::vector<int32_t> *state, std::vector<int32_t> *it)
{
    cudaError_t e = cudaSuccess;
    if (state) {
        state->resize(c->n_cases);
        e = cudaMemcpyAsync(state->data(), c->case_state, c->n_cases * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            c->stream);
    }
    if (it && e == cudaSuccess) {
        it->resize(c->n_cases);
        e = cudaMemcpyAsync(it->data(), c->case_it, c->n_cases * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the case counters");
    return LSKUM_OK;
}

// Room for `need` norms per case ([n_cases][cap] rows, copied row by row).
lskum_status ensure_hist(lskum_ctx *c, int32_t need)
{
    if (need <= c->hist_cap) return LSKUM_OK;
    int32_t cap = c->hist_cap;
    while (cap < need) cap *= 2;
    double *h = nullptr, *h4 = nullptr;
    cudaError_t e = cudaMalloc(&h, (size_t)c->n_cases * cap * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h4, (size_t)c->n_cases * cap * 4 * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(h);
        return cuda_fail(c, e, "cudaMalloc(history)");
    }
    e = cudaMemcpy2DAsync(h, cap * sizeof(double), c->hist, c->hist_cap * sizeof(double),
                          c->hist_cap * sizeof(double), c->n_cases, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(h4, 4 * cap * sizeof(double), c->hist4, 4 * c->hist_cap * sizeof(double),
                              4 * c->hist_cap * sizeof(double), c->n_cases, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(h);
        cudaFree(h4);
        return cuda_fail(c, e, "copying the history");
    }
    for (auto &p : c->arena.ptrs) {
        if (p == c->hist) {
            cudaFree(p);
            p = h;
        } else if (p == c->hist4) {
            cudaFree(p);
            p = h4;
        }
    }
    c->hist = h;
    c->hist4 = h4;
    c->hist_cap = cap;
    Ctrl hc{};
    lskum_status s = read_ctrl(c, &hc);  // the device copy points at the new arrays
    if (s == LSKUM_OK) s = write_ctrl(c, hc);
    return s;
}

lskum_status finish_state(lskum_ctx *c, bool reset_hist, bool project);

lskum_status state_from_conserved(lskum_ctx *c, const double *Ucaller, bool reset_hist, bool project)
{
    // caller order, contiguous: one copy straight from the caller's memory,
    // then the reordering into the internal structure of arrays on the device
    // (or, where the device reads pageable host memory, the reordering kernel
    // reads the caller's array itself; finish_state synchronises before the
    // call returns, so the caller may reuse the array)
    const int32_t n = c->n;
    cudaError_t e = join_user(c);
    const double *src = Ucaller;
    if (!c->host_direct) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->dscratch, Ucaller, 4 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream);
        src = c->dscratch;
    }
    if (e == cudaSuccess) e = launch_from_caller(src, c->ld, n, c->dev.inv, c->dev.set[c->cur].U, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "setting the state");
    return finish_state(c, reset_hist, project);
}

// The conserved state of the current set was written on the device: derive
// q and the per-point quantities (with the wall projection when `project`:
// a state built from primitives or predicted; a conserved checkpoint is
// taken as given, since re-projecting a projected state can move its last
// bit), check it, and reset the counters (all of them with reset_hist).
lskum_status finish_state(lskum_ctx *c, bool reset_hist, bool project)
{
    // a new state: the increments restart from zero (the revised LU-SGS
    // lags its S term on the previous increment)
    cudaError_t e = cudaMemsetAsync(c->dev.dU, 0, 4 * (size_t)c->ld * sizeof(double), c->stream);
    if (e == cudaSuccess && c->dev.dUf)
        e = cudaMemsetAsync(c->dev.dUf, 0, 4 * (size_t)c->ld * sizeof(float), c->stream);
    if (e == cudaSuccess) e = launch_reset_ctrl(c->ctrl, c->stream);
    if (e == cudaSuccess) e = launch_init_state(c->dev, c->cur, project, c->stream);
    Ctrl h{};
    if (e != cudaSuccess) return cuda_fail(c, e, "setting the state");
    lskum_status s = read_ctrl(c, &h);
    if (s != LSKUM_OK) return s;
    if (h.error) return fail(c, LSKUM_ERR_NONPOSITIVE, "non-physical state at point %d", c->perm[h.bad_point]);
    if (reset_hist) {
        h.it = 0;
        c->hist_bound = 0;
    }
    h.stop = h.error = 0;
    h.bad_point = 0x7fffffff;
    s = reset_cases(c, reset_hist, true);
    if (s == LSKUM_OK) s = write_ctrl(c, h);
    if (s != LSKUM_OK) return s;
    e = release_user(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "ordering the caller's stream");
    return LSKUM_OK;
}

}  // namespace

extern "C" {

lskum_status lskum_set_state(lskum_ctx *c, const double *rho, const double *u, const double *v, const double *p)
{
    if (!c || !rho || !u || !v || !p) return c ? fail(c, LSKUM_ERR_ARG, "NULL argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    std::vector<double> U(4 * (size_t)c->n);
    for (int32_t k = 0; k < c->n; k++) {
        if (!(rho[k] > 0.0) || !(p[k] > 0.0) || !std::isfinite(rho[k]) || !std::isfinite(p[k]) ||
            !std::isfinite(u[k]) || !std::isfinite(v[k]))
            return fail(c, LSKUM_ERR_NONPOSITIVE, "non-physical input state at point %d", k);
        host_prim_to_cons(rho[k], u[k], v[k], p[k], &U[4 * (size_t)k]);
    }
    return state_from_conserved(c, U.data(), true, true);
}

lskum_status lskum_set_conserved(lskum_ctx *c, const double *U)
{
    if (!c || !U) return c ? fail(c, LSKUM_ERR_ARG, "NULL argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    return state_from_conserved(c, U, false, false);
}

// Asynchronous part of lskum_run: enqueue max_iters graph launches.
lskum_status lskum_enqueue(lskum_ctx *c, int32_t max_iters, double target_drop)
{
    if (!c || max_iters < 0) return c ? fail(c, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    // no host round trip: the history bound is kept on the host and the
    // control block is prepared by a kernel ahead of the graph launches
    if (c->hist_bound + max_iters > INT32_MAX / 8) return fail(c, LSKUM_ERR_ARG, "history too long");
    lskum_status s = ensure_hist(c, (int32_t)(c->hist_bound + max_iters));
    if (s != LSKUM_OK) return s;
    c->hist_bound += max_iters;
    cudaError_t e = join_user(c);
    if (e == cudaSuccess) e = launch_prep_run(c->ctrl, target_drop, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "preparing the run");
    c->cur_base = c->cur;
    int par = c->cur;
    for (int32_t i = 0; i < max_iters && e == cudaSuccess; i++) {
        e = cudaGraphLaunch(c->graph[par], c->stream);
        par ^= 1;
    }
    if (e == cudaSuccess) e = release_user(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "enqueueing iterations");
    c->pending = true;
    return LSKUM_OK;
}

lskum_status lskum_wait(lskum_ctx *c, int32_t *iters_done)
{
    if (iters_done) *iters_done = 0;
    if (!c) return LSKUM_ERR_ARG;
    if (!c->pending) return LSKUM_OK;
    c->pending = false;
    Ctrl h{};
    lskum_status s = read_ctrl(c, &h);
    if (s != LSKUM_OK) return s;
    int32_t done = h.it - h.it_start;  // iterations started (k_begin)
    if (h.error) done -= 1;            // the failed iteration's update was not applied
    c->cur = (c->cur_base + done) & 1;
    if (iters_done) *iters_done = done;
    if (h.error == LSKUM_ERR_NONPOSITIVE)
        return fail(c, LSKUM_ERR_NONPOSITIVE, "non-physical update at point %d in iteration %d",
                    c->perm[h.bad_point], h.it);
    if (h.error == LSKUM_ERR_DIVERGED)
        return fail(c, LSKUM_ERR_DIVERGED, "residual norm of case %d not finite in iteration %d", -1 - h.bad_point,
                    h.it);
    if (h.error) return fail(c, LSKUM_ERR_CUDA, "device error %d", h.error);
    return LSKUM_OK;
}

lskum_status lskum_run(lskum_ctx *c, int32_t max_iters, double target_drop, int32_t *iters_done)
{
    lskum_status s = lskum_enqueue(c, max_iters, target_drop);
    if (s != LSKUM_OK) {
        if (iters_done) *iters_done = 0;
        return s;
    }
    return lskum_wait(c, iters_done);
}

void *lskum_stream(lskum_ctx *c)
{
    return c ? (void *)c->stream : nullptr;
}

// Copy a per-point field to the host in caller order: reordered on the
// device (from `comps` rows of stride ld when stride is 0, else `comps`
// values of point k at stride * k; FP32 when srcf is given), then one
// contiguous copy.
static lskum_status download_to(lskum_ctx *c, const double *src, const float *srcf, int comps, int stride,
                                double *out)
{
    const size_t bytes = (size_t)comps * c->n * sizeof(double);
    cudaError_t e = launch_to_caller(src, srcf, comps, stride, c->ld, c->n, c->dev.inv,
                                     c->host_direct ? out : c->dscratch, c->stream);
    if (e == cudaSuccess && !c->host_direct)
        e = cudaMemcpyAsync(out, c->dscratch, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy D2H");
    return LSKUM_OK;
}

static lskum_status download(lskum_ctx *c, const double *src, int comps, std::vector<double> &out, int stride = 0)
{
    out.resize((size_t)comps * c->n);
    return download_to(c, src, nullptr, comps, stride, out.data());
}

lskum_status lskum_get_field(lskum_ctx *c, int32_t field, double *out)
{
    if (!c || !out) return c ? fail(c, LSKUM_ERR_ARG, "NULL argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    const Dev &d = c->dev;
    const int K = d.K & 1;
    const double *src = nullptr;
    int comps = 4, stride = 0;
    switch (field) {
    case LSKUM_FIELD_U: src = d.set[c->cur].U; break;
    case LSKUM_FIELD_Q: src = d.set[c->cur].q; break;
    case LSKUM_FIELD_QX: src = d.gq[K]; stride = 8; break;
    case LSKUM_FIELD_QY: src = d.gq[K] + 4; stride = 8; break;
    case LSKUM_FIELD_R: src = d.R; break;
    case LSKUM_FIELD_D: src = d.D; comps = 1; break;
    case LSKUM_FIELD_DUS: src = d.dUs; stride = 4; break;
    case LSKUM_FIELD_DU: src = d.dU; stride = 4; break;
    default: return fail(c, LSKUM_ERR_ARG, "unknown field %d", field);
    }
    const float *srcf = nullptr;
    if (d.precision && (field == LSKUM_FIELD_DUS || field == LSKUM_FIELD_DU))
        srcf = field == LSKUM_FIELD_DUS ? d.dUsf : d.dUf;  // FP32 increments of the mixed-precision sweeps
    return download_to(c, src, srcf, comps, stride, out);
}

// Order stream `waiter` after the work already enqueued on `waited`.
static cudaError_t order_after(lskum_ctx *c, cudaStream_t waiter, cudaStream_t waited)
{
    cudaError_t e = cudaEventRecord(c->ev, waited);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(waiter, c->ev, 0);
    return e;
}

lskum_status lskum_get_field_dev(lskum_ctx *c, int32_t field, double *out_dev, void *cuda_stream)
{
    if (!c || !out_dev) return c ? fail(c, LSKUM_ERR_ARG, "NULL argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    const Dev &d = c->dev;
    const int K = d.K & 1;
    const double *src = nullptr;
    const float *srcf = nullptr;
    int comps = 4, stride = 0;
    switch (field) {
    case LSKUM_FIELD_U: src = d.set[c->cur].U; break;
    case LSKUM_FIELD_Q: src = d.set[c->cur].q; break;
    case LSKUM_FIELD_QX: src = d.gq[K]; stride = 8; break;
    case LSKUM_FIELD_QY: src = d.gq[K] + 4; stride = 8; break;
    case LSKUM_FIELD_R: src = d.R; break;
    case LSKUM_FIELD_D: src = d.D; comps = 1; break;
    case LSKUM_FIELD_DUS: src = d.dUs; srcf = d.precision ? d.dUsf : nullptr; stride = 4; break;
    case LSKUM_FIELD_DU: src = d.dU; srcf = d.precision ? d.dUf : nullptr; stride = 4; break;
    default: return fail(c, LSKUM_ERR_ARG, "unknown field %d", field);
    }
    cudaStream_t us = (cudaStream_t)cuda_stream;
    cudaError_t e = order_after(c, c->stream, us);
    if (e == cudaSuccess) e = launch_to_caller(src, srcf, comps, stride, c->ld, c->n, d.inv, out_dev, c->stream);
    if (e == cudaSuccess) e = order_after(c, us, c->stream);
    return e == cudaSuccess ? LSKUM_OK : cuda_fail(c, e, "field to device memory");
}

lskum_status lskum_set_conserved_dev(lskum_ctx *c, const double *U_dev, void *cuda_stream)
{
    if (!c || !U_dev) return c ? fail(c, LSKUM_ERR_ARG, "NULL argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    cudaStream_t us = (cudaStream_t)cuda_stream;
    cudaError_t e = order_after(c, c->stream, us);
    if (e == cudaSuccess) e = launch_from_caller(U_dev, c->ld, c->n, c->dev.inv, c->dev.set[c->cur].U, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "state from device memory");
    lskum_status s = finish_state(c, false, false);
    if (s != LSKUM_OK) return s;
    e = order_after(c, us, c->stream);
    return e == cudaSuccess ? LSKUM_OK : cuda_fail(c, e, "ordering the caller's stream");
}

lskum_status lskum_get_state(lskum_ctx *c, double *rho, double *u, double *v, double *p)
{
    if (!c || !rho || !u || !v || !p) return c ? fail(c, LSKUM_ERR_ARG, "NULL argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    std::vector<double> U;
    lskum_status s = download(c, c->dev.set[c->cur].U, 4, U);
    if (s != LSKUM_OK) return s;
    for (int32_t k = 0; k < c->n; k++) {
        const double r = U[4 * (size_t)k];
        rho[k] = r;
        u[k] = U[4 * (size_t)k + 1] / r;
        v[k] = U[4 * (size_t)k + 2] / r;
        p[k] = 0.4 * (U[4 * (size_t)k + 3] - 0.5 * r * (u[k] * u[k] + v[k] * v[k]));
    }
    return LSKUM_OK;
}

lskum_status lskum_get_case_residuals(lskum_ctx *c, int32_t cs, double *hist, int32_t cap, int32_t *n)
{
    if (!c || !n || cap < 0 || (cap > 0 && !hist) || cs < 0 || cs >= (c ? c->n_cases : 0))
        return c ? fail(c, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    std::vector<int32_t> its;
    lskum_status s = read_case_arrays(c, nullptr, &its);
    if (s != LSKUM_OK) return s;
    *n = std::min(its[cs], c->hist_cap);
    const int32_t m = std::min(cap, *n);
    if (m > 0) {
        cudaError_t e = cudaMemcpyAsync(hist, c->hist + (size_t)cs * c->hist_cap, m * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy history");
    }
    return LSKUM_OK;
}

lskum_status lskum_get_case_residuals4(lskum_ctx *c, int32_t cs, double *hist4, int32_t cap, int32_t *n)
{
    if (!c || !n || cap < 0 || (cap > 0 && !hist4) || cs < 0 || cs >= (c ? c->n_cases : 0))
        return c ? fail(c, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    std::vector<int32_t> its;
    lskum_status s = read_case_arrays(c, nullptr, &its);
    if (s != LSKUM_OK) return s;
    *n = std::min(its[cs], c->hist_cap);
    const int32_t m = std::min(*n, cap);
    if (m > 0) {
        cudaError_t e = cudaMemcpyAsync(hist4, c->hist4 + (size_t)cs * c->hist_cap * 4, 4 * (size_t)m * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "reading the residual history");
    }
    return LSKUM_OK;
}

lskum_status lskum_get_residuals(lskum_ctx *c, double *hist, int32_t cap, int32_t *n)
{
    return lskum_get_case_residuals(c, 0, hist, cap, n);
}

lskum_status lskum_get_case_forces(lskum_ctx *c, int32_t cs, double *cl, double *cd)
{
    if (!c || !cl || !cd || cs < 0 || cs >= c->n_cases) return c ? fail(c, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    std::vector<double> U;
    lskum_status s = download(c, c->dev.set[c->cur].U, 4, U);
    if (s != LSKUM_OK) return s;
    std::vector<int32_t> w;
    for (int32_t p = c->case_off[cs]; p < c->case_off[cs + 1]; p++)
        if (c->flag[p] == LSKUM_WALL) w.push_back(p);
    *cl = 0.0;
    *cd = 0.0;
    const int32_t nw = (int32_t)w.size();
    if (nw < 3) return LSKUM_OK;
    double area2 = 0.0;
    for (int32_t k = 0; k < nw; k++) {
        const int32_t a = w[k], b = w[(k + 1) % nw];
        area2 += c->x[a] * c->y[b] - c->x[b] * c->y[a];
    }
    const double orient = area2 > 0.0 ? 1.0 : -1.0;
    const double pinf = 1.0 / 1.4;
    double Fx = 0.0, Fy = 0.0;
    for (int32_t k = 0; k < nw; k++) {
        const int32_t a = w[(k + nw - 1) % nw], m = w[k], b = w[(k + 1) % nw];
        const double ex = 0.5 * (c->x[b] - c->x[a]), ey = 0.5 * (c->y[b] - c->y[a]);
        const double r = U[4 * (size_t)m];
        const double uu = U[4 * (size_t)m + 1] / r, vv = U[4 * (size_t)m + 2] / r;
        const double pr = 0.4 * (U[4 * (size_t)m + 3] - 0.5 * r * (uu * uu + vv * vv));
        Fx -= (pr - pinf) * orient * ey;
        Fy -= (pr - pinf) * (-orient * ex);
    }
    const double al = c->case_aoa[cs] * M_PI / 180.0;
    const double qinf = 0.5 * c->case_mach[cs] * c->case_mach[cs];
    *cl = (Fy * std::cos(al) - Fx * std::sin(al)) / qinf;
    *cd = (Fx * std::cos(al) + Fy * std::sin(al)) / qinf;
    return LSKUM_OK;
}

lskum_status lskum_get_forces(lskum_ctx *c, double *cl, double *cd)
{
    return lskum_get_case_forces(c, 0, cl, cd);
}

lskum_status lskum_get_case_info(lskum_ctx *c, int32_t cs, int32_t *first_point, int32_t *n_points,
                                 int32_t *iters, int32_t *stopped, int32_t *status, int32_t *bad_point)
{
    if (!c || cs < 0 || cs >= c->n_cases) return c ? fail(c, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    std::vector<int32_t> st, its;
    lskum_status s = read_case_arrays(c, &st, &its);
    int32_t err = 0, bad = 0x7fffffff;
    cudaError_t e = cudaSuccess;
    if (s == LSKUM_OK) {
        e = cudaMemcpyAsync(&err, c->case_err + cs, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&bad, c->case_bad + cs, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = cuda_fail(c, e, "reading the case status");
    }
    if (s != LSKUM_OK) return s;
    if (first_point) *first_point = c->case_off[cs];
    if (n_points) *n_points = c->case_off[cs + 1] - c->case_off[cs];
    if (iters) *iters = its[cs];
    if (stopped) *stopped = st[cs] != kRunning;
    if (status) *status = err;
    if (bad_point) *bad_point = (err == LSKUM_ERR_NONPOSITIVE && bad >= 0 && bad < c->n) ? c->perm[bad] : -1;
    return LSKUM_OK;
}

lskum_status lskum_time_phases(lskum_ctx *c, int32_t reps, double *ms)
{
    if (!c || reps < 1 || !ms) return c ? fail(c, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    Ctrl h{};
    lskum_status s = read_ctrl(c, &h);
    std::vector<int32_t> its;
    if (s == LSKUM_OK) s = read_case_arrays(c, nullptr, &its);
    if (s != LSKUM_OK) return s;
    s = ensure_hist(c, *std::max_element(its.begin(), its.end()) + reps);
    if (s != LSKUM_OK) return s;
    c->hist_bound += reps;
    h.stop = h.error = 0;
    h.target = 0.0;
    s = reset_cases(c, false, false);
    if (s == LSKUM_OK) s = write_ctrl(c, h);
    if (s != LSKUM_OK) return s;
    cudaError_t e = cudaSuccess;
    cudaEvent_t ev[7];
    for (auto &x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const Dev &d = c->dev;
    for (int32_t r = 0; r < reps && e == cudaSuccess; r++) {
        const int cur = c->cur;
        for (int ph = 0; ph < 6 && e == cudaSuccess; ph++) {
            e = cudaEventRecord(ev[ph], c->stream);
            if (e == cudaSuccess) e = launch_phase(d, c->launch, cur, ph, c->n_levels, c->lvl_beg.data(),
                                                   c->lvl_act_end.data(), c->lvl_end.data(), c->stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev[6], c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[6]);
        for (int ph = 0; ph < 6 && e == cudaSuccess; ph++) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[ph], ev[ph + 1]);
            acc[ph] += t;
        }
        c->cur ^= 1;
    }
    for (auto &x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_fail(c, e, "timing phases");
    Ctrl h2{};
    s = read_ctrl(c, &h2);
    if (s != LSKUM_OK) return s;
    if (h2.error) {
        c->cur ^= 1;
        return fail(c, (lskum_status)h2.error, "iteration failed while timing phases");
    }
    for (int ph = 0; ph < 6; ph++) ms[ph] = acc[ph] / reps;
    return LSKUM_OK;
}

lskum_status lskum_autotune(lskum_ctx *c, int32_t trial_iters, int32_t *tpp, int32_t *sweep_lanes, double *ms_per_iter)
{
    if (!c || trial_iters < 1) return c ? fail(c, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    // save the state set (device copies, so the restored state is bitwise
    // the same), the counters and the histories; every trial is restored
    const size_t ld = c->ld;
    const size_t bytes_d = (8 * ld + (size_t)kPrimStride * ld) * sizeof(double);
    const size_t bytes_f = c->dev.set[0].primf ? (size_t)kPrimStride * ld * sizeof(float) : 0;
    const size_t bytes_inc = 4 * ld * sizeof(double) + (c->dev.dUf ? 4 * ld * sizeof(float) : 0);
    char *save = nullptr;
    cudaError_t e = cudaMalloc(&save, bytes_d + bytes_f + bytes_inc);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(autotune save)");
    struct Free {
        char *p;
        ~Free() { cudaFree(p); }
    } free_save{save};
    auto copy_set = [&](bool to_save) -> cudaError_t {
        const StateSet &st = c->dev.set[c->cur];
        // the state set and the last increments (the revised LU-SGS lags on them)
        char *parts[6] = {(char *)st.U, (char *)st.q, (char *)st.prim, (char *)st.primf, (char *)c->dev.dU,
                          (char *)c->dev.dUf};
        const size_t sz[6] = {4 * ld * sizeof(double), 4 * ld * sizeof(double),
                              (size_t)kPrimStride * ld * sizeof(double), bytes_f, 4 * ld * sizeof(double),
                              c->dev.dUf ? 4 * ld * sizeof(float) : 0};
        size_t off = 0;
        cudaError_t ee = cudaSuccess;
        for (int i = 0; i < 6 && ee == cudaSuccess; i++) {
            if (!sz[i]) continue;
            ee = to_save ? cudaMemcpyAsync(save + off, parts[i], sz[i], cudaMemcpyDeviceToDevice, c->stream)
                         : cudaMemcpyAsync(parts[i], save + off, sz[i], cudaMemcpyDeviceToDevice, c->stream);
            off += sz[i];
        }
        return ee;
    };
    e = copy_set(true);
    if (e != cudaSuccess) return cuda_fail(c, e, "saving the state");
    lskum_status s = LSKUM_OK;
    Ctrl h0{};
    s = read_ctrl(c, &h0);
    std::vector<int32_t> st0, it0;
    if (s == LSKUM_OK) s = read_case_arrays(c, &st0, &it0);
    if (s == LSKUM_OK) s = ensure_hist(c, *std::max_element(it0.begin(), it0.end()) + trial_iters + 2);
    if (s != LSKUM_OK) return s;
    std::vector<double> hist0(c->n_cases), hist((size_t)c->n_cases * c->hist_cap);
    e = cudaMemcpyAsync(hist0.data(), c->case_hist0, c->n_cases * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hist.data(), c->hist, hist.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "saving the state");
    const int cap0 = c->hist_cap;
    auto restore = [&]() -> lskum_status {
        cudaError_t ee = copy_set(false);
        if (ee == cudaSuccess)
            ee = cudaMemcpyAsync(c->case_it, it0.data(), c->n_cases * sizeof(int32_t),
                                         cudaMemcpyHostToDevice, c->stream);
        if (ee == cudaSuccess)
            ee = cudaMemcpyAsync(c->case_state, st0.data(), c->n_cases * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 c->stream);
        if (ee == cudaSuccess)
            ee = cudaMemcpyAsync(c->case_hist0, hist0.data(), c->n_cases * sizeof(double), cudaMemcpyHostToDevice,
                                 c->stream);
        if (ee == cudaSuccess)
            ee = cudaMemcpy2DAsync(c->hist, c->hist_cap * sizeof(double), hist.data(), cap0 * sizeof(double),
                                   cap0 * sizeof(double), c->n_cases, cudaMemcpyHostToDevice, c->stream);
        if (ee == cudaSuccess) ee = cudaStreamSynchronize(c->stream);
        if (ee != cudaSuccess) return cuda_fail(c, ee, "restoring the state");
        Ctrl h = h0;
        h.stop = h.error = 0;
        return write_ctrl(c, h);
    };
    const Launch orig = c->launch;
    Launch best = orig;
    double best_ms = 1e300;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
    for (int tp : {1, 2, 4, 8}) {
        for (int gl : {2, 4, 8, 32}) {
            if (gl == 32 && !c->pk_ok) continue;
            c->launch.tpp = tp;
            c->launch.sweep_lanes = gl;
            s = build_graphs(c);
            int32_t warm = 0;
            if (s == LSKUM_OK) s = lskum_run(c, 1, 0.0, &warm);  // warm-up
            if (s == LSKUM_OK) s = lskum_enqueue(c, 0, 0.0);     // sets up the control block
            if (s == LSKUM_OK) s = lskum_wait(c, nullptr);
            if (s != LSKUM_OK) break;
            const int32_t it_start = h0.it + warm;
            int par = c->cur;
            e = cudaEventRecord(e0, c->stream);
            for (int32_t i = 0; i < trial_iters && e == cudaSuccess; i++, par ^= 1)
                e = cudaGraphLaunch(c->graph[par], c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                s = cuda_fail(c, e, "timing a launch shape");
                break;
            }
            Ctrl hc{};
            s = read_ctrl(c, &hc);
            if (s != LSKUM_OK) break;
            c->cur = (c->cur + (hc.it - it_start)) & 1;  // trial iterations that ran
            if (warm == 1 && !hc.error && !hc.stop && hc.it - it_start == trial_iters &&
                ms / trial_iters < best_ms) {
                best_ms = ms / trial_iters;
                best = c->launch;
            }
            s = restore();
            if (s != LSKUM_OK) break;
        }
        if (s != LSKUM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->launch = s == LSKUM_OK ? best : orig;
    lskum_status s2 = build_graphs(c);
    if (s == LSKUM_OK) s = restore();
    if (s != LSKUM_OK) return s;
    if (s2 != LSKUM_OK) return s2;
    if (tpp) *tpp = c->launch.tpp;
    if (sweep_lanes) *sweep_lanes = c->launch.sweep_lanes;
    if (ms_per_iter) *ms_per_iter = best_ms;
    return LSKUM_OK;
}

lskum_status lskum_get_order(lskum_ctx *c, int32_t *colour, int32_t *order, int32_t *n_colours)
{
    if (!c) return LSKUM_ERR_ARG;
    if (colour) std::memcpy(colour, c->colour.data(), c->n * sizeof(int32_t));
    if (order) std::memcpy(order, c->canon_order.data(), c->n * sizeof(int32_t));
    if (n_colours) *n_colours = c->n_colours;
    return LSKUM_OK;
}

lskum_status lskum_set_host_io(lskum_ctx *c, int32_t direct)
{
    if (!c || (direct != 0 && direct != 1)) return c ? fail(c, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    if (direct && !c->host_direct_ok)
        return fail(c, LSKUM_ERR_ARG, "the device cannot access pageable host memory directly");
    c->host_direct = direct == 1;
    return LSKUM_OK;
}

lskum_status lskum_get_host_io(lskum_ctx *c, int32_t *direct, int32_t *supported)
{
    if (!c) return LSKUM_ERR_ARG;
    if (direct) *direct = c->host_direct ? 1 : 0;
    if (supported) *supported = c->host_direct_ok ? 1 : 0;
    return LSKUM_OK;
}

lskum_status lskum_get_info(lskum_ctx *c, int32_t *n_points, int32_t *n_colours, int32_t *launches_per_iter)
{
    if (!c) return LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    if (n_points) *n_points = c->n;
    if (n_colours) *n_colours = c->n_colours;
    if (launches_per_iter) *launches_per_iter = c->launches_per_iter;
    return LSKUM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// what the warm-start network needs from a context (lskum_mlp_internal.h)
// ---------------------------------------------------------------------------
namespace lskum {

CtxHost ctx_host(lskum_ctx *c)
{
    return CtxHost{c->n, c->n_cases, c->perm.data(), c->inv.data(), c->flag.data(), c->case_of_caller.data()};
}

lskum_status ctx_fail(lskum_ctx *c, lskum_status s, const char *msg)
{
    return fail(c, s, "%s", msg);
}

lskum_status ctx_case_status(lskum_ctx *c, std::vector<int32_t> &status)
{
    status.assign(c->n_cases, 0);
    cudaError_t e = cudaMemcpyAsync(status.data(), c->case_err, c->n_cases * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? LSKUM_OK : cuda_fail(c, e, "reading the case status");
}

lskum_status ctx_mlp_view(lskum_ctx *c, MlpView *v)
{
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    const int32_t n = c->n, ld = c->ld;
    if (!c->mx) {
        std::vector<float> hx(ld, 0.f), hy(ld, 0.f), cm(c->n_cases), ca(c->n_cases);
        std::vector<double> cU(4 * (size_t)c->n_cases), cuv(2 * (size_t)c->n_cases);
        for (int32_t b = 0; b < c->n_cases; b++) {
            host_free_stream(c, b, &cuv[2 * b], &cuv[2 * b + 1]);
            host_prim_to_cons(1.0, cuv[2 * b], cuv[2 * b + 1], 1.0 / 1.4, &cU[4 * b]);
        }
        for (int32_t k = 0; k < n; k++) {
            hx[k] = (float)c->x[c->perm[k]];
            hy[k] = (float)c->y[c->perm[k]];
        }
        for (int32_t b = 0; b < c->n_cases; b++) {
            cm[b] = (float)c->case_mach[b];
            ca[b] = (float)c->case_aoa[b];
        }
        // per case: its wall polygon (wall points in caller order, closed)
        std::vector<float4> seg;
        std::vector<int32_t> seg_off(c->n_cases + 1, 0);
        for (int32_t b = 0; b < c->n_cases; b++) {
            std::vector<int32_t> w;
            for (int32_t p = c->case_off[b]; p < c->case_off[b + 1]; p++)
                if (c->flag[p] == LSKUM_WALL) w.push_back(p);
            for (size_t i = 0; i < w.size(); i++) {
                const int32_t a = w[i], q = w[(i + 1) % w.size()];
                seg.push_back(make_float4((float)c->x[a], (float)c->y[a], (float)c->x[q], (float)c->y[q]));
            }
            seg_off[b + 1] = (int32_t)seg.size();
        }
        Arena &A = c->arena;
        float *dx = A.alloc<float>(ld), *dy = A.alloc<float>(ld), *dw = A.alloc<float>(ld);
        float *dm = A.alloc<float>(c->n_cases), *da = A.alloc<float>(c->n_cases);
        double *dU = A.alloc<double>(4 * (size_t)c->n_cases), *duv = A.alloc<double>(2 * (size_t)c->n_cases);
        float4 *dseg = A.alloc<float4>(seg.size());
        int32_t *doff = A.alloc<int32_t>(seg_off.size());
        if (A.err != cudaSuccess) return cuda_fail(c, A.err, "cudaMalloc(network geometry)");
        cudaError_t e = cudaMemcpyAsync(dx, hx.data(), ld * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dy, hy.data(), ld * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dm, cm.data(), c->n_cases * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(da, ca.data(), c->n_cases * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dU, cU.data(), cU.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(duv, cuv.data(), cuv.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && !seg.empty())
            e = cudaMemcpyAsync(dseg, seg.data(), seg.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(doff, seg_off.data(), seg_off.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(dw, 0, ld * sizeof(float), c->stream);
        if (e == cudaSuccess) e = launch_wall_distance(dx, dy, c->dev.case_of, n, dseg, doff, dw, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the host vectors go out of scope
        if (e != cudaSuccess) return cuda_fail(c, e, "network geometry");
        c->mx = dx;
        c->my = dy;
        c->mdw = dw;
        c->mcase_mach = dm;
        c->mcase_aoa = da;
        c->mcase_Uinf = dU;
        c->mcase_uv = duv;
    }
    v->n = n;
    v->ld = ld;
    v->n_cases = c->n_cases;
    v->x = c->mx;
    v->y = c->my;
    v->dwall = c->mdw;
    v->flag = c->dev.flag;
    v->case_of = c->dev.case_of;
    v->case_mach = c->mcase_mach;
    v->case_aoa = c->mcase_aoa;
    v->case_Uinf = c->mcase_Uinf;
    v->case_uv = c->mcase_uv;
    v->U = c->dev.set[c->cur].U;
    v->stream = c->stream;
    return LSKUM_OK;
}

lskum_status ctx_state_written(lskum_ctx *c)
{
    return finish_state(c, true, true);
}

// First residual norm of every case at the current state: one iteration's
// q-derivatives, residual and norm (no sweeps, no update), then the counters
// are cleared.  A norm that is not finite comes back as infinity.
lskum_status ctx_case_norms(lskum_ctx *c, std::vector<double> &norms)
{
    Ctrl h{};
    lskum_status s = read_ctrl(c, &h);
    if (s == LSKUM_OK) s = reset_cases(c, true, true);
    if (s != LSKUM_OK) return s;
    h.it = 0;
    h.stop = h.error = 0;
    h.target = 0.0;
    h.bad_point = 0x7fffffff;
    s = write_ctrl(c, h);
    if (s != LSKUM_OK) return s;
    cudaError_t e = cudaSuccess;
    for (int ph = 0; ph < 3 && e == cudaSuccess; ph++)
        e = launch_phase(c->dev, c->launch, c->cur, ph, c->n_levels, c->lvl_beg.data(), c->lvl_act_end.data(),
                         c->lvl_end.data(), c->stream);
    norms.assign(c->n_cases, 0.0);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(norms.data(), sizeof(double), c->hist, c->hist_cap * sizeof(double), sizeof(double),
                              c->n_cases, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "residual norms");
    for (auto &x : norms)
        if (!std::isfinite(x)) x = INFINITY;
    s = read_ctrl(c, &h);
    if (s == LSKUM_OK) s = reset_cases(c, true, true);
    if (s != LSKUM_OK) return s;
    h.it = 0;
    h.stop = h.error = 0;
    h.bad_point = 0x7fffffff;
    return write_ctrl(c, h);
}

}  // namespace lskum

extern "C" {

lskum_status lskum_get_wall_distance(lskum_ctx *c, double *d)
{
    if (!c || !d) return c ? fail(c, LSKUM_ERR_ARG, "NULL argument") : LSKUM_ERR_ARG;
    MlpView v{};
    lskum_status s = ctx_mlp_view(c, &v);
    if (s != LSKUM_OK) return s;
    std::vector<float> dw(c->ld);
    cudaError_t e = cudaMemcpyAsync(dw.data(), v.dwall, c->ld * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the wall distance");
    for (int32_t p = 0; p < c->n; p++) d[p] = dw[c->inv[p]];
    return LSKUM_OK;
}

lskum_status lskum_selftest_fpint(int32_t op, const double *a, const double *b, double *out, int32_t n)
{
    if (op < 0 || op > 3 || n < 0 || (n > 0 && (!a || !out || ((op == 0 || op == 3) && !b))))
        return LSKUM_ERR_ARG;
    if (n == 0) return LSKUM_OK;
    double *da = nullptr, *db = nullptr, *dout = nullptr;
    const size_t bytes = (size_t)n * sizeof(double);
    cudaError_t e = cudaMalloc(&da, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&db, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&dout, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(da, a, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = b ? cudaMemcpy(db, b, bytes, cudaMemcpyHostToDevice) : cudaMemset(db, 0, bytes);
    if (e == cudaSuccess) e = launch_selftest_fpint(op, da, db, dout, n, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
    cudaFree(da);
    cudaFree(db);
    cudaFree(dout);
    return e == cudaSuccess ? LSKUM_OK : LSKUM_ERR_CUDA;
}

lskum_status lskum_set_launch_shape(lskum_ctx *c, int32_t tpp, int32_t sweep_lanes)
{
    if (!c) return LSKUM_ERR_ARG;
    if ((tpp != 1 && tpp != 2 && tpp != 4 && tpp != 8) ||
        (sweep_lanes != 2 && sweep_lanes != 4 && sweep_lanes != 8 && !(sweep_lanes == 32 && c->pk_ok)))
        return fail(c, LSKUM_ERR_ARG, "launch shape %d, %d not supported", tpp, sweep_lanes);
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    c->launch.tpp = tpp;
    c->launch.sweep_lanes = sweep_lanes;
    return build_graphs(c);
}

lskum_status lskum_set_start_iters(lskum_ctx *c, int32_t first_order_iters)
{
    if (!c || first_order_iters < 0) return c ? fail(c, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    if (c->pending) return fail(c, LSKUM_ERR_ARG, "an enqueued run has not been waited for");
    c->opts.first_order_iters = first_order_iters;
    c->dev.first_order = first_order_iters;
    return build_graphs(c);
}

}  // extern "C"
