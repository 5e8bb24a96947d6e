/*
 * FastDOG oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of what the GPU path
 * computes, written directly from the paper (Abbas & Swoboda, "FastDOG: Fast
 * Discrete Optimization on GPU", CVPR 2022):
 *
 *   - BDD construction for one linear row a^T x in [L, U]      (Def. 4, Ex. 1)
 *   - presolve of forced variables / always-true rows           (a forced variable
 *     would give infinite min-marginal differences, so it is fixed first)
 *   - shortest paths and min-marginals on a weighted BDD        (Eq. 6, Alg. 3, Alg. 4)
 *   - parallel deferred min-marginal averaging, lifted form     (Alg. 1, Eq. 5, Prop. 1 proof)
 *   - the final deferred add-back                               (Alg. 1, last loop)
 *   - perturbation primal rounding                              (Alg. 2)
 *   - the objective c^T x
 *
 * Only tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load this library.  It shares no code, header or constant with the CUDA
 * library, and the CUDA library never calls it.
 *
 * Conventions
 *   - Everything is double precision and strictly sequential: BDDs in
 *     construction order (= row order), layers in the order Alg. 1 states.
 *   - The dual state is kept in the lifted representation of the Appendix
 *     (a pair hi = lambda^{j,1}_i, lo = lambda^{j,0}_i per slot); the plain
 *     multiplier is lambda = hi - lo.
 *   - Where the paper leaves a detail open: M-bar is refreshed after every
 *     pass; the final step of Alg. 1 adds the averaged deferred differences
 *     back; the lifted update subtracts the positive parts and adds their
 *     averages; arcs leaving layer i carry lambda_i (pinned by Fig. 3).
 *
 * Status codes: 0 ok, -1 invalid input, -2 out of memory / too large,
 * -3 infeasible, -5 wrong call order, -7 rounding did not converge.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EINFEASIBLE (-3)
#define ORC_ESTATE (-5)
#define ORC_ENOCONVERGE (-7)

#define TOP (-1)
#define BOT (-2)

#define MAX_STATES_PER_ROW (1 << 22)

/* ------------------------------------------------------------------------- */
/* One BDD (Def. 4): layer t holds nodes [lstart[t], lstart[t+1]); node 0 is  */
/* the root; lo/hi are the 0-arc and 1-arc successors (node index in layer   */
/* t+1, or TOP / BOT).                                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    int k;       /* number of variables = layers */
    int nn;      /* number of nodes */
    int *lstart; /* k + 1 entries */
    int *lo, *hi;
} bdd_t;

static void bdd_free(bdd_t *b) {
    free(b->lstart);
    free(b->lo);
    free(b->hi);
    memset(b, 0, sizeof(*b));
}

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* index of s in sorted array v[0..n), or -1 */
static int find_i64(const int64_t *v, int n, int64_t s) {
    int a = 0, b = n - 1;
    while (a <= b) {
        int m = (a + b) / 2;
        if (v[m] == s) return m;
        if (v[m] < s) a = m + 1; else b = m - 1;
    }
    return -1;
}

/*
 * Build the ordered BDD of { x in {0,1}^k : L <= sum_t a[t] x[t] <= U }
 * (Ex. 1 turns one ILP row into one subproblem; Def. 4 fixes the layered
 * form).  Top-down, a node of layer t is a reachable partial sum of the first
 * t terms; a partial sum from which no completion can reach [L, U] goes to
 * BOT.  Bottom-up, a node whose two arcs both reach BOT becomes BOT and nodes
 * of one layer with equal (lo, hi) are merged, which gives the reduced
 * (canonical, no isomorphic subgraphs) form the paper's remark mentions.
 * Layers are never skipped.  Returns ORC_EINFEASIBLE if the set is empty.
 */
static int build_row_bdd(int k, const int64_t *a, int haveL, int64_t L, int haveU, int64_t U, bdd_t *out) {
    memset(out, 0, sizeof(*out));
    if (k <= 0) return ORC_EINVAL;
    int64_t *rmin = calloc(k + 1, sizeof(int64_t)), *rmax = calloc(k + 1, sizeof(int64_t));
    int64_t **st = calloc(k + 1, sizeof(int64_t *)); /* states per layer */
    int *ns = calloc(k + 1, sizeof(int));
    int **clo = calloc(k, sizeof(int *)), **chi = calloc(k, sizeof(int *));
    int rc = ORC_OK;
    if (!rmin || !rmax || !st || !ns || !clo || !chi) { rc = ORC_ENOMEM; goto done; }
    for (int t = k - 1; t >= 0; --t) {
        rmin[t] = rmin[t + 1] + (a[t] < 0 ? a[t] : 0);
        rmax[t] = rmax[t + 1] + (a[t] > 0 ? a[t] : 0);
    }
#define LIVE(t, s) ((!haveL || (s) + rmax[t] >= L) && (!haveU || (s) + rmin[t] <= U))
#define SAT(s) ((!haveL || (s) >= L) && (!haveU || (s) <= U))
    if (!LIVE(0, (int64_t)0)) { rc = ORC_EINFEASIBLE; goto done; }
    st[0] = malloc(sizeof(int64_t));
    st[0][0] = 0;
    ns[0] = 1;
    int64_t total = 1;
    for (int t = 0; t < k; ++t) {
        int n = ns[t];
        clo[t] = malloc(sizeof(int) * n);
        chi[t] = malloc(sizeof(int) * n);
        if (!clo[t] || !chi[t]) { rc = ORC_ENOMEM; goto done; }
        if (t + 1 == k) {
            for (int v = 0; v < n; ++v) {
                clo[t][v] = SAT(st[t][v]) ? TOP : BOT;
                chi[t][v] = SAT(st[t][v] + a[t]) ? TOP : BOT;
            }
            break;
        }
        int64_t *cand = malloc(sizeof(int64_t) * 2 * (size_t)n);
        if (!cand) { rc = ORC_ENOMEM; goto done; }
        int nc = 0;
        for (int v = 0; v < n; ++v) {
            int64_t s0 = st[t][v], s1 = st[t][v] + a[t];
            if (LIVE(t + 1, s0)) cand[nc++] = s0;
            if (LIVE(t + 1, s1)) cand[nc++] = s1;
        }
        qsort(cand, nc, sizeof(int64_t), cmp_i64);
        int nu = 0;
        for (int q = 0; q < nc; ++q)
            if (nu == 0 || cand[nu - 1] != cand[q]) cand[nu++] = cand[q];
        st[t + 1] = cand;
        ns[t + 1] = nu;
        total += nu;
        if (total > MAX_STATES_PER_ROW) { rc = ORC_ENOMEM; goto done; }
        for (int v = 0; v < n; ++v) {
            int64_t s0 = st[t][v], s1 = st[t][v] + a[t];
            clo[t][v] = LIVE(t + 1, s0) ? find_i64(cand, nu, s0) : BOT;
            chi[t][v] = LIVE(t + 1, s1) ? find_i64(cand, nu, s1) : BOT;
        }
    }
#undef LIVE
#undef SAT
    {
        /* bottom-up reduction: map[t][v] = reduced id of state v in layer t (or BOT) */
        int **map = calloc(k, sizeof(int *));
        int *rn = calloc(k, sizeof(int));              /* reduced node count per layer */
        int **rlo = calloc(k, sizeof(int *)), **rhi = calloc(k, sizeof(int *));
        if (!map || !rn || !rlo || !rhi) { rc = ORC_ENOMEM; free(map); free(rn); free(rlo); free(rhi); goto done; }
        for (int t = k - 1; t >= 0; --t) {
            int n = ns[t];
            map[t] = malloc(sizeof(int) * n);
            rlo[t] = malloc(sizeof(int) * n);
            rhi[t] = malloc(sizeof(int) * n);
            for (int v = 0; v < n; ++v) {
                int l = clo[t][v], h = chi[t][v];
                if (t + 1 < k) {
                    if (l >= 0) l = map[t + 1][l];
                    if (h >= 0) h = map[t + 1][h];
                }
                if (l == BOT && h == BOT) { map[t][v] = BOT; continue; }
                int found = -1;
                for (int r = 0; r < rn[t]; ++r)
                    if (rlo[t][r] == l && rhi[t][r] == h) { found = r; break; }
                if (found < 0) {
                    found = rn[t]++;
                    rlo[t][found] = l;
                    rhi[t][found] = h;
                }
                map[t][v] = found;
            }
        }
        if (map[0][0] == BOT) {
            rc = ORC_EINFEASIBLE;
        } else {
            /* layer 0 has exactly one state, so rn[0] == 1 and the root is node 0 */
            int nn = 0;
            for (int t = 0; t < k; ++t) nn += rn[t];
            out->k = k;
            out->nn = nn;
            out->lstart = malloc(sizeof(int) * (k + 1));
            out->lo = malloc(sizeof(int) * nn);
            out->hi = malloc(sizeof(int) * nn);
            int off = 0;
            for (int t = 0; t < k; ++t) {
                out->lstart[t] = off;
                int nxt = off + rn[t];
                for (int r = 0; r < rn[t]; ++r) {
                    int l = rlo[t][r], h = rhi[t][r];
                    out->lo[off + r] = l >= 0 ? nxt + l : l;
                    out->hi[off + r] = h >= 0 ? nxt + h : h;
                }
                off = nxt;
            }
            out->lstart[k] = off;
        }
        for (int t = 0; t < k; ++t) { free(map[t]); free(rlo[t]); free(rhi[t]); }
        free(map); free(rn); free(rlo); free(rhi);
    }
done:
    if (st) for (int t = 0; t <= k; ++t) free(st[t]);
    if (clo) for (int t = 0; t < k; ++t) { free(clo[t]); }
    if (chi) for (int t = 0; t < k; ++t) { free(chi[t]); }
    free(st); free(ns); free(clo); free(chi); free(rmin); free(rmax);
    return rc;
}

/* the BDD of the full cube {0,1}^k: one node per layer, both arcs to the next */
static int bdd_is_full_cube(const bdd_t *b) {
    for (int t = 0; t < b->k; ++t) {
        if (b->lstart[t + 1] - b->lstart[t] != 1) return 0;
        int v = b->lstart[t];
        if (b->lo[v] != b->hi[v] || b->lo[v] == BOT) return 0;
    }
    return 1;
}

/* 1 if every node of layer t has its 1-arc to BOT (x_t forced to 0), 2 if every
   0-arc goes to BOT (forced to 1), 0 otherwise.  Every node of a reduced BDD
   built above lies on a root-TOP path, so this is exact. */
static int bdd_forced(const bdd_t *b, int t) {
    int all_hi_bot = 1, all_lo_bot = 1;
    for (int v = b->lstart[t]; v < b->lstart[t + 1]; ++v) {
        if (b->hi[v] != BOT) all_hi_bot = 0;
        if (b->lo[v] != BOT) all_lo_bot = 0;
    }
    return all_hi_bot ? 1 : (all_lo_bot ? 2 : 0);
}

/* ------------------------------------------------------------------------- */
/* problem                                                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n;
    double *c;
    int8_t *fixed;   /* -1: in some BDD; 0/1: fixed by presolve; 2: in no row (free) */
    double const_lb; /* sum over fixed c_i x_i plus sum over free min(c_i, 0) */
    double const_obj_fixed;
    int m;           /* number of BDDs (rows kept after presolve) */
    int *row;        /* original row of each BDD */
    bdd_t *bdd;
    int64_t *slot0;  /* first slot of each BDD; slot = one (BDD j, variable i in I_j) */
    int64_t *node0;  /* first node of each BDD in the global node arrays */
    int64_t S, N;
    int *svar;       /* variable of each slot */
    double *hi, *lo; /* lifted multipliers lambda^{j,1}_i, lambda^{j,0}_i */
    double *spf, *spb;
    int spf_valid, spb_valid; /* labels consistent with the current (hi, lo) */
    int *cnt;        /* |J_i| */
    double *D0, *D1, *Db0, *Db1;
    /* row data kept for presolve-free feasibility checks in tests */
} orc_problem;

static double pos(double x) { return x > 0 ? x : 0; }

/* presolve: repeatedly substitute fixed variables into rows,
   drop rows whose feasible set is the full cube, fix variables that a row
   forces, until nothing changes. */
static int presolve_and_build(orc_problem *p, int n_rows, const int64_t *row_ptr, const int32_t *col,
                              const int32_t *coef, const int8_t *sense, const int64_t *rhs) {
    int n = p->n;
    int8_t *alive = malloc(n_rows ? n_rows : 1);
    for (int j = 0; j < n_rows; ++j) alive[j] = 1;
    for (int i = 0; i < n; ++i) p->fixed[i] = -1;
    int64_t maxlen = 1;
    for (int j = 0; j < n_rows; ++j)
        if (row_ptr[j + 1] - row_ptr[j] > maxlen) maxlen = row_ptr[j + 1] - row_ptr[j];
    int *vv = malloc(sizeof(int) * maxlen);
    int64_t *aa = malloc(sizeof(int64_t) * maxlen);
    int rc = ORC_OK;
    int changed = 1;
    while (changed && rc == ORC_OK) {
        changed = 0;
        for (int j = 0; j < n_rows && rc == ORC_OK; ++j) {
            if (!alive[j]) continue;
            int k = 0;
            int64_t shift = 0;
            for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q) {
                if (coef[q] == 0) continue;
                int i = col[q];
                if (p->fixed[i] == 0 || p->fixed[i] == 1) { shift += (int64_t)coef[q] * p->fixed[i]; continue; }
                /* insertion into ascending variable order (Alg. 1 visits I_j ascending) */
                int pos_ = k++;
                while (pos_ > 0 && vv[pos_ - 1] > i) { vv[pos_] = vv[pos_ - 1]; aa[pos_] = aa[pos_ - 1]; --pos_; }
                vv[pos_] = i;
                aa[pos_] = coef[q];
            }
            int haveL = sense[j] >= 0, haveU = sense[j] <= 0;
            int64_t b = rhs[j] - shift;
            if (k == 0) {
                if ((haveL && 0 < b) || (haveU && 0 > b)) rc = ORC_EINFEASIBLE;
                alive[j] = 0;
                continue;
            }
            bdd_t B;
            int r = build_row_bdd(k, aa, haveL, b, haveU, b, &B);
            if (r != ORC_OK) { rc = r; break; }
            if (bdd_is_full_cube(&B)) {
                alive[j] = 0;
            } else {
                for (int t = 0; t < k; ++t) {
                    int f = bdd_forced(&B, t);
                    if (f) { p->fixed[vv[t]] = (int8_t)(f == 1 ? 0 : 1); changed = 1; }
                }
                if (changed) { /* the row is re-examined with its fixed variables substituted */ }
            }
            bdd_free(&B);
        }
    }
    if (rc != ORC_OK) { free(alive); free(vv); free(aa); return rc; }

    /* final BDDs of the surviving rows */
    int m = 0;
    for (int j = 0; j < n_rows; ++j) m += alive[j];
    p->m = m;
    p->row = malloc(sizeof(int) * (m ? m : 1));
    p->bdd = calloc(m ? m : 1, sizeof(bdd_t));
    p->slot0 = malloc(sizeof(int64_t) * (m + 1));
    p->node0 = malloc(sizeof(int64_t) * (m + 1));
    int **vars = calloc(m ? m : 1, sizeof(int *));
    int jj = 0;
    int64_t S = 0, N = 0;
    for (int j = 0; j < n_rows && rc == ORC_OK; ++j) {
        if (!alive[j]) continue;
        int k = 0;
        int64_t shift = 0;
        for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q) {
            if (coef[q] == 0) continue;
            int i = col[q];
            if (p->fixed[i] == 0 || p->fixed[i] == 1) { shift += (int64_t)coef[q] * p->fixed[i]; continue; }
            int pos_ = k++;
            while (pos_ > 0 && vv[pos_ - 1] > i) { vv[pos_] = vv[pos_ - 1]; aa[pos_] = aa[pos_ - 1]; --pos_; }
            vv[pos_] = i;
            aa[pos_] = coef[q];
        }
        int haveL = sense[j] >= 0, haveU = sense[j] <= 0;
        int64_t b = rhs[j] - shift;
        rc = build_row_bdd(k, aa, haveL, b, haveU, b, &p->bdd[jj]);
        if (rc != ORC_OK) break;
        p->row[jj] = j;
        vars[jj] = malloc(sizeof(int) * k);
        memcpy(vars[jj], vv, sizeof(int) * k);
        p->slot0[jj] = S;
        p->node0[jj] = N;
        S += k;
        N += p->bdd[jj].nn;
        ++jj;
    }
    free(alive); free(vv); free(aa);
    if (rc != ORC_OK) {
        for (int q = 0; q < jj; ++q) free(vars[q]);
        free(vars);
        return rc;
    }
    p->slot0[m] = S;
    p->node0[m] = N;
    p->S = S;
    p->N = N;
    p->svar = malloc(sizeof(int) * (S ? S : 1));
    for (int q = 0; q < m; ++q) {
        memcpy(p->svar + p->slot0[q], vars[q], sizeof(int) * p->bdd[q].k);
        free(vars[q]);
    }
    free(vars);
    return ORC_OK;
}

void orc_destroy(orc_problem *p);

/* Build the problem: presolve, one BDD per remaining row, and the
   initialisation lambda^j_i = c_i / |J_i| (Alg. 1 text), i.e. hi = c_i/|J_i|,
   lo = 0 in the lifted form, with M-bar = 0. */
int orc_create(int n_vars, const double *cost, int n_rows, const int64_t *row_ptr, const int32_t *col,
               const int32_t *coef, const int8_t *sense, const int64_t *rhs, orc_problem **out) {
    *out = NULL;
    if (n_vars < 0 || n_rows < 0) return ORC_EINVAL;
    for (int j = 0; j < n_rows; ++j) {
        if (row_ptr[j + 1] < row_ptr[j]) return ORC_EINVAL;
        if (sense[j] < -1 || sense[j] > 1) return ORC_EINVAL;
        for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q) {
            if (col[q] < 0 || col[q] >= n_vars) return ORC_EINVAL;
            for (int64_t r = row_ptr[j]; r < q; ++r)
                if (col[r] == col[q]) return ORC_EINVAL; /* duplicate variable in a row */
        }
    }
    for (int i = 0; i < n_vars; ++i)
        if (!isfinite(cost[i])) return ORC_EINVAL;
    orc_problem *p = calloc(1, sizeof(orc_problem));
    p->n = n_vars;
    p->c = malloc(sizeof(double) * (n_vars ? n_vars : 1));
    memcpy(p->c, cost, sizeof(double) * n_vars);
    p->fixed = malloc(n_vars ? n_vars : 1);
    int rc = presolve_and_build(p, n_rows, row_ptr, col, coef, sense, rhs);
    if (rc != ORC_OK) { orc_destroy(p); return rc; }
    int n = n_vars;
    p->cnt = calloc(n ? n : 1, sizeof(int));
    for (int64_t s = 0; s < p->S; ++s) p->cnt[p->svar[s]]++;
    p->const_lb = 0;
    p->const_obj_fixed = 0;
    for (int i = 0; i < n; ++i) {
        if (p->fixed[i] == 0 || p->fixed[i] == 1) {
            p->const_lb += p->c[i] * p->fixed[i];
            p->const_obj_fixed += p->c[i] * p->fixed[i];
        } else if (p->cnt[i] == 0) {
            p->fixed[i] = 2; /* in no row: x_i = [c_i < 0], bound += min(c_i, 0) */
            p->const_lb += p->c[i] < 0 ? p->c[i] : 0;
        }
    }
    int64_t S = p->S ? p->S : 1, N = p->N ? p->N : 1;
    p->hi = malloc(sizeof(double) * S);
    p->lo = malloc(sizeof(double) * S);
    p->spf = malloc(sizeof(double) * N);
    p->spb = malloc(sizeof(double) * N);
    p->D0 = calloc(n ? n : 1, sizeof(double));
    p->D1 = calloc(n ? n : 1, sizeof(double));
    p->Db0 = calloc(n ? n : 1, sizeof(double));
    p->Db1 = calloc(n ? n : 1, sizeof(double));
    for (int64_t s = 0; s < p->S; ++s) {
        int i = p->svar[s];
        p->hi[s] = p->c[i] / p->cnt[i];
        p->lo[s] = 0.0;
    }
    p->spb_valid = p->spf_valid = 0;
    *out = p;
    return ORC_OK;
}

void orc_destroy(orc_problem *p) {
    if (!p) return;
    if (p->bdd) for (int j = 0; j < p->m; ++j) bdd_free(&p->bdd[j]);
    free(p->bdd); free(p->row); free(p->slot0); free(p->node0); free(p->svar);
    free(p->hi); free(p->lo); free(p->spf); free(p->spb); free(p->cnt);
    free(p->D0); free(p->D1); free(p->Db0); free(p->Db1); free(p->c); free(p->fixed);
    free(p);
}

/* ------------------------------------------------------------------------- */
/* shortest paths on one weighted BDD with given per-layer arc costs          */
/* (0-arc of layer t costs w0[t], 1-arc costs w1[t]; arcs leave layer t).     */
/* ------------------------------------------------------------------------- */
static double succ(const double *d, int v) { return v == TOP ? 0.0 : (v == BOT ? INFINITY : d[v]); }

static void sp_forward(const bdd_t *b, const double *w0, const double *w1, double *f) {
    for (int v = 0; v < b->nn; ++v) f[v] = INFINITY;
    f[0] = 0.0;
    for (int t = 0; t < b->k; ++t)
        for (int v = b->lstart[t]; v < b->lstart[t + 1]; ++v) {
            if (b->lo[v] >= 0 && f[v] + w0[t] < f[b->lo[v]]) f[b->lo[v]] = f[v] + w0[t];
            if (b->hi[v] >= 0 && f[v] + w1[t] < f[b->hi[v]]) f[b->hi[v]] = f[v] + w1[t];
        }
}

static void sp_backward(const bdd_t *b, const double *w0, const double *w1, double *g) {
    for (int t = b->k - 1; t >= 0; --t)
        for (int v = b->lstart[t]; v < b->lstart[t + 1]; ++v) {
            double a0 = succ(g, b->lo[v]) + w0[t], a1 = succ(g, b->hi[v]) + w1[t];
            g[v] = a0 < a1 ? a0 : a1;
        }
}

/* Eq. 6: m^beta_t = min over v in layer t with s^beta(v) != BOT of
   SP(r,v) + cost of the beta-arc + SP(s^beta(v), TOP). */
static void layer_min_marginals(const bdd_t *b, int t, const double *f, const double *g, double w0, double w1,
                                double *m0, double *m1) {
    double a = INFINITY, c = INFINITY;
    for (int v = b->lstart[t]; v < b->lstart[t + 1]; ++v) {
        if (b->lo[v] != BOT) { double x = f[v] + w0 + succ(g, b->lo[v]); if (x < a) a = x; }
        if (b->hi[v] != BOT) { double x = f[v] + w1 + succ(g, b->hi[v]); if (x < c) c = x; }
    }
    *m0 = a;
    *m1 = c;
}

/* ------------------------------------------------------------------------- */
/* Alg. 1 in the lifted form of the Appendix.                                 */
/* ------------------------------------------------------------------------- */

/* full sweeps at the current (hi, lo): SP(v, TOP), resp. SP(r, v), for every node */
static void refresh_spb(orc_problem *p) {
    for (int j = 0; j < p->m; ++j)
        sp_backward(&p->bdd[j], p->lo + p->slot0[j], p->hi + p->slot0[j], p->spb + p->node0[j]);
    p->spb_valid = 1;
}
static void refresh_spf(orc_problem *p) {
    for (int j = 0; j < p->m; ++j)
        sp_forward(&p->bdd[j], p->lo + p->slot0[j], p->hi + p->slot0[j], p->spf + p->node0[j]);
    p->spf_valid = 1;
}

/*
 * One pass of Alg. 1 over all BDDs (sequentially; the paper runs them in
 * parallel, which is equivalent because each BDD only reads M-bar from the
 * previous pass).  forward = 1: layers in ascending order, shortest paths from
 * the root updated incrementally (Alg. 3) against SP(., TOP) of the previous
 * backward pass; forward = 0: descending order (Alg. 4) against SP(r, .) of
 * the previous forward pass.  Per slot (Eq. 5 in lifted form):
 *     d = m^1 - m^0
 *     hi -= omega * max(d, 0);        lo -= omega * max(-d, 0)
 *     hi += omega * Dbar1_i / |J_i|;  lo += omega * Dbar0_i / |J_i|
 * and D^beta_i accumulates max(+-d, 0).  After the pass M-bar <- M.
 * M_out (may be NULL) receives d per slot.
 */
static void run_pass(orc_problem *p, int forward, double omega, double *M_out) {
    int n = p->n;
    for (int i = 0; i < n; ++i) { p->D0[i] = 0; p->D1[i] = 0; }
    if (forward && !p->spb_valid) refresh_spb(p);
    if (!forward && !p->spf_valid) refresh_spf(p);
    for (int j = 0; j < p->m; ++j) {
        const bdd_t *b = &p->bdd[j];
        double *hi = p->hi + p->slot0[j], *lo = p->lo + p->slot0[j];
        double *f = p->spf + p->node0[j], *g = p->spb + p->node0[j];
        const int *vars = p->svar + p->slot0[j];
        if (forward) {
            for (int v = 0; v < b->nn; ++v) f[v] = INFINITY;
            f[0] = 0.0;
        }
        for (int q = 0; q < b->k; ++q) {
            int t = forward ? q : b->k - 1 - q;
            int i = vars[t];
            double m0, m1;
            layer_min_marginals(b, t, f, g, lo[t], hi[t], &m0, &m1);
            double d = m1 - m0;
            hi[t] -= omega * pos(d);
            lo[t] -= omega * pos(-d);
            hi[t] += omega * p->Db1[i] / p->cnt[i];
            lo[t] += omega * p->Db0[i] / p->cnt[i];
            p->D1[i] += pos(d);
            p->D0[i] += pos(-d);
            if (M_out) M_out[p->slot0[j] + t] = d;
            if (forward) {
                /* Alg. 3: shortest paths from the root into layer t+1 with the updated costs */
                for (int v = b->lstart[t]; v < b->lstart[t + 1]; ++v) {
                    if (b->lo[v] >= 0 && f[v] + lo[t] < f[b->lo[v]]) f[b->lo[v]] = f[v] + lo[t];
                    if (b->hi[v] >= 0 && f[v] + hi[t] < f[b->hi[v]]) f[b->hi[v]] = f[v] + hi[t];
                }
            } else {
                /* Alg. 4: shortest paths to TOP for layer t with the updated costs */
                for (int v = b->lstart[t]; v < b->lstart[t + 1]; ++v) {
                    double a0 = succ(g, b->lo[v]) + lo[t], a1 = succ(g, b->hi[v]) + hi[t];
                    g[v] = a0 < a1 ? a0 : a1;
                }
            }
        }
    }
    /* M-bar <- M */
    for (int i = 0; i < n; ++i) { p->Db0[i] = p->D0[i]; p->Db1[i] = p->D1[i]; }
    /* a forward pass leaves SP(r, .) current and SP(., TOP) stale, and vice versa */
    p->spf_valid = forward;
    p->spb_valid = !forward;
}

/* E(lambda^{j,1}, lambda^{j,0}) of BDD j by a full backward sweep at the given costs */
static double bdd_energy(const orc_problem *p, int j, const double *w0, const double *w1, double *scratch) {
    sp_backward(&p->bdd[j], w0, w1, scratch);
    return scratch[0];
}

static int64_t max_nodes(const orc_problem *p) {
    int64_t mx = 1;
    for (int j = 0; j < p->m; ++j) if (p->bdd[j].nn > mx) mx = p->bdd[j].nn;
    return mx;
}
static int64_t max_layers(const orc_problem *p) {
    int64_t mx = 1;
    for (int j = 0; j < p->m; ++j) if (p->bdd[j].k > mx) mx = p->bdd[j].k;
    return mx;
}

/* lower bounds at the current state (nothing is modified):
   running  = sum_j E(hi^j, lo^j) + constant          (lifted bound, Prop. 1 proof)
   feasible = the same after the final add-back of Alg. 1. */
int orc_lower_bounds(const orc_problem *p, double omega, double *lb_running, double *lb_feasible) {
    double *scr = malloc(sizeof(double) * max_nodes(p));
    int64_t K = max_layers(p);
    double *w0 = malloc(sizeof(double) * K), *w1 = malloc(sizeof(double) * K);
    double run = p->const_lb, fea = p->const_lb;
    for (int j = 0; j < p->m; ++j) {
        const double *hi = p->hi + p->slot0[j], *lo = p->lo + p->slot0[j];
        const int *vars = p->svar + p->slot0[j];
        run += bdd_energy(p, j, lo, hi, scr);
        for (int t = 0; t < p->bdd[j].k; ++t) {
            int i = vars[t];
            w1[t] = hi[t] + omega * p->Db1[i] / p->cnt[i];
            w0[t] = lo[t] + omega * p->Db0[i] / p->cnt[i];
        }
        fea += bdd_energy(p, j, w0, w1, scr);
    }
    free(scr); free(w0); free(w1);
    if (lb_running) *lb_running = run;
    if (lb_feasible) *lb_feasible = fea;
    return ORC_OK;
}

/* E(hi^j, lo^j) of every BDD at the current state (the terms of the running bound) */
int orc_energies(const orc_problem *p, double *E) {
    double *scr = malloc(sizeof(double) * max_nodes(p));
    for (int j = 0; j < p->m; ++j) E[j] = bdd_energy(p, j, p->lo + p->slot0[j], p->hi + p->slot0[j], scr);
    free(scr);
    return ORC_OK;
}

/* one pass; exposed so that tests can check Prop. 1 after every pass */
int orc_pass(orc_problem *p, int forward, double omega, double *M_out) {
    if (!(omega > 0 && omega <= 1)) return ORC_EINVAL;
    run_pass(p, forward, omega, M_out);
    return ORC_OK;
}

/* k iterations of Alg. 1 (ascending pass, then descending pass); lb_trace[t]
   (may be NULL) gets the running lifted bound after iteration t. */
int orc_iterate(orc_problem *p, int k, double omega, double *lb_trace) {
    if (!(omega > 0 && omega <= 1) || k < 0) return ORC_EINVAL;
    for (int t = 0; t < k; ++t) {
        run_pass(p, 1, omega, NULL);
        run_pass(p, 0, omega, NULL);
        if (lb_trace) {
            double lb = p->const_lb;
            for (int j = 0; j < p->m; ++j) lb += p->spb[p->node0[j]]; /* SP(r, TOP) after the backward pass */
            lb_trace[t] = lb;
        }
    }
    return ORC_OK;
}

/*
 * The serial min-marginal averaging of Eq. 4 (the prior scheme the paper
 * contrasts with Alg. 1): variables are visited one at a time, in ascending
 * index order and then in descending order (one iteration); for variable i
 * the min-marginal differences M_ij of all its copies are computed at the
 * current multipliers (Eq. 6, from full shortest-path sweeps of each BDD) and
 * every copy is set to lambda^j_i - M_ij + (1/|J_i|) sum_k M_ik, after which
 * all copies share one difference and sum_j lambda^j_i is unchanged.  The
 * state is the plain multipliers (lo = 0, no deferred differences).
 * lb_trace[t] (may be NULL) gets sum_j E_j + constant after iteration t.
 */
int orc_iterate_serial(orc_problem *p, int k, double *lb_trace) {
    if (k < 0) return ORC_EINVAL;
    int64_t S = p->S;
    int n = p->n;
    /* plain multipliers; no deferred state */
    for (int64_t s = 0; s < S; ++s) { p->hi[s] -= p->lo[s]; p->lo[s] = 0.0; }
    for (int i = 0; i < n; ++i) { p->D0[i] = p->D1[i] = p->Db0[i] = p->Db1[i] = 0.0; }
    p->spf_valid = p->spb_valid = 0;
    /* copies of each variable (ascending slots) and the BDD of each slot */
    int64_t *vs0 = calloc(n + 1, sizeof(int64_t));
    int64_t *vsl = malloc(sizeof(int64_t) * (S ? S : 1));
    int *sbdd = malloc(sizeof(int) * (S ? S : 1));
    for (int64_t s = 0; s < S; ++s) vs0[p->svar[s] + 1]++;
    for (int i = 0; i < n; ++i) vs0[i + 1] += vs0[i];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) fill[i] = vs0[i];
    for (int64_t s = 0; s < S; ++s) vsl[fill[p->svar[s]]++] = s;
    for (int j = 0; j < p->m; ++j)
        for (int t = 0; t < p->bdd[j].k; ++t) sbdd[p->slot0[j] + t] = j;
    int64_t NN = max_nodes(p), K = max_layers(p);
    double *f = malloc(sizeof(double) * NN), *g = malloc(sizeof(double) * NN);
    double *w0 = calloc(K > 0 ? K : 1, sizeof(double)), *w1 = malloc(sizeof(double) * (K > 0 ? K : 1));
    int cmax = 0;
    for (int i = 0; i < n; ++i) if (vs0[i + 1] - vs0[i] > cmax) cmax = (int)(vs0[i + 1] - vs0[i]);
    double *M = malloc(sizeof(double) * (cmax > 0 ? cmax : 1));
    for (int it = 0; it < k; ++it) {
        for (int dir = 0; dir < 2; ++dir) {
            for (int q = 0; q < n; ++q) {
                int i = dir == 0 ? q : n - 1 - q;
                int c = (int)(vs0[i + 1] - vs0[i]);
                if (c == 0) continue;
                double sum = 0.0;
                for (int r = 0; r < c; ++r) {
                    int64_t s = vsl[vs0[i] + r];
                    int j = sbdd[s];
                    const bdd_t *b = &p->bdd[j];
                    int64_t s0 = p->slot0[j];
                    for (int t = 0; t < b->k; ++t) { w0[t] = 0.0; w1[t] = p->hi[s0 + t]; }
                    sp_forward(b, w0, w1, f);
                    sp_backward(b, w0, w1, g);
                    double m0, m1;
                    int t = (int)(s - s0);
                    layer_min_marginals(b, t, f, g, w0[t], w1[t], &m0, &m1);
                    M[r] = m1 - m0;
                    sum += M[r];
                }
                double avg = sum / c;
                for (int r = 0; r < c; ++r) p->hi[vsl[vs0[i] + r]] += avg - M[r];
            }
        }
        if (lb_trace) {
            double lb = p->const_lb;
            double *scr = f;
            for (int j = 0; j < p->m; ++j) lb += bdd_energy(p, j, p->lo + p->slot0[j], p->hi + p->slot0[j], scr);
            lb_trace[it] = lb;
        }
    }
    free(vs0); free(vsl); free(sbdd); free(fill); free(f); free(g); free(w0); free(w1); free(M);
    return ORC_OK;
}

/* final step of Alg. 1: add the deferred differences back (averaged) */
int orc_addback(orc_problem *p, double omega) {
    for (int64_t s = 0; s < p->S; ++s) {
        int i = p->svar[s];
        p->hi[s] += omega * p->Db1[i] / p->cnt[i];
        p->lo[s] += omega * p->Db0[i] / p->cnt[i];
    }
    for (int i = 0; i < p->n; ++i) { p->Db0[i] = 0; p->Db1[i] = 0; }
    p->spb_valid = p->spf_valid = 0;
    return ORC_OK;
}

/* min-marginals at lambda = hi - lo (the plain, non-lifted multipliers) for
   every slot, in slot order, by full forward and backward sweeps and Eq. 6 */
int orc_min_marginals(const orc_problem *p, double *m0, double *m1) {
    int64_t NN = max_nodes(p), K = max_layers(p);
    double *f = malloc(sizeof(double) * NN), *g = malloc(sizeof(double) * NN);
    double *w0 = calloc(K, sizeof(double)), *w1 = malloc(sizeof(double) * K);
    for (int j = 0; j < p->m; ++j) {
        const bdd_t *b = &p->bdd[j];
        int64_t s0 = p->slot0[j];
        for (int t = 0; t < b->k; ++t) { w0[t] = 0.0; w1[t] = p->hi[s0 + t] - p->lo[s0 + t]; }
        sp_forward(b, w0, w1, f);
        sp_backward(b, w0, w1, g);
        for (int t = 0; t < b->k; ++t) layer_min_marginals(b, t, f, g, w0[t], w1[t], m0 + s0 + t, m1 + s0 + t);
    }
    free(f); free(g); free(w0); free(w1);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Alg. 2: perturbation primal rounding                                       */
/* ------------------------------------------------------------------------- */

/* SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014), applied to
   one counter value: the first output of a SplitMix64 generator seeded with x. */
static uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t x) { return splitmix64(x); }

/* u uniform in [0, 1) from SplitMix64(seed ^ round << 32 ^ variable), returned
   as 2u - 1 in [-1, 1); Alg. 2 scales it by delta to draw r from [-delta, delta) */
double orc_uniform_pm1(uint64_t seed, int round, int var) {
    uint64_t h = splitmix64(seed ^ ((uint64_t)(uint32_t)round << 32) ^ (uint64_t)(uint32_t)var);
    double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    return 2.0 * u - 1.0;
}

/*
 * Alg. 2.  Starts with the final add-back of Alg. 1, computes all M_ij, and
 * while some variable's differences do not all share one strict nonzero sign
 * (all-zero differences count as disagreement: they fix no assignment),
 * perturbs every variable by the cases of Alg. 2 with r uniform in
 * [-delta, delta) (the conflict case with sum_j M_ij = 0 takes sign(r)),
 * multiplies delta by alpha, re-optimises with `kr` iterations of Alg. 1 from
 * M-bar = 0 followed by the add-back, and recomputes M.  At agreement
 * x_i = [M_ij < 0].
 * Output: x (n bytes), rounds used, objective c^T x, and `margin` = the smallest
 * |M_ij| (and |sum_j M_ij| of conflicting variables) met in any round's
 * decisions, which bounds how robust the decisions are to rounding error.
 */
int orc_round(orc_problem *p, double omega, double delta, double alpha, int kr, int max_rounds, uint64_t seed,
              uint8_t *x, int *rounds_out, double *obj_out, double *margin_out) {
    orc_addback(p, omega);
    int64_t S = p->S;
    double *m0 = malloc(sizeof(double) * (S ? S : 1)), *m1 = malloc(sizeof(double) * (S ? S : 1));
    double *M = malloc(sizeof(double) * (S ? S : 1));
    int n = p->n;
    /* per-variable slot lists */
    int64_t *vs0 = calloc(n + 1, sizeof(int64_t));
    int64_t *vsl = malloc(sizeof(int64_t) * (S ? S : 1));
    for (int64_t s = 0; s < S; ++s) vs0[p->svar[s] + 1]++;
    for (int i = 0; i < n; ++i) vs0[i + 1] += vs0[i];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) fill[i] = vs0[i];
    for (int64_t s = 0; s < S; ++s) vsl[fill[p->svar[s]]++] = s;
    double margin = INFINITY;
    int round = 0, rc = ORC_OK;
    for (;;) {
        orc_min_marginals(p, m0, m1);
        for (int64_t s = 0; s < S; ++s) M[s] = m1[s] - m0[s];
        int disagree = 0;
        for (int i = 0; i < n && !disagree; ++i) {
            if (vs0[i] == vs0[i + 1]) continue;
            int npos = 0, nneg = 0, c = (int)(vs0[i + 1] - vs0[i]);
            for (int64_t q = vs0[i]; q < vs0[i + 1]; ++q) { npos += M[vsl[q]] > 0; nneg += M[vsl[q]] < 0; }
            if (!(npos == c || nneg == c)) disagree = 1;
        }
        for (int64_t s = 0; s < S; ++s) if (fabs(M[s]) < margin) margin = fabs(M[s]);
        if (!disagree) break;
        if (round >= max_rounds) { rc = ORC_ENOCONVERGE; break; }
        for (int i = 0; i < n; ++i) {
            if (vs0[i] == vs0[i + 1]) continue;
            int npos = 0, nneg = 0, nzero = 0, c = (int)(vs0[i + 1] - vs0[i]);
            double sum = 0.0;
            for (int64_t q = vs0[i]; q < vs0[i + 1]; ++q) {
                double v = M[vsl[q]];
                npos += v > 0; nneg += v < 0; nzero += v == 0;
                sum += v;
            }
            /* Alg. 2 draws r uniformly from [-delta, delta] and pushes by r * delta */
            double r = orc_uniform_pm1(seed, round, i) * delta;
            double pert;
            if (npos == c) pert = delta;
            else if (nneg == c) pert = -delta;
            else if (nzero == c) pert = r * delta;
            else {
                double sg = sum > 0 ? 1.0 : (sum < 0 ? -1.0 : (r >= 0 ? 1.0 : -1.0));
                pert = sg * fabs(r) * delta;
                if (fabs(sum) < margin) margin = fabs(sum);
            }
            for (int64_t q = vs0[i]; q < vs0[i + 1]; ++q) p->hi[vsl[q]] += pert;
        }
        delta *= alpha;
        /* re-optimise: Alg. 1 from M-bar = 0, then its final add-back */
        for (int i = 0; i < n; ++i) { p->Db0[i] = 0; p->Db1[i] = 0; }
        p->spb_valid = p->spf_valid = 0;
        orc_iterate(p, kr, omega, NULL);
        orc_addback(p, omega);
        ++round;
    }
    double obj = 0.0;
    for (int i = 0; i < n; ++i) {
        uint8_t xi;
        if (p->fixed[i] == 0 || p->fixed[i] == 1) xi = (uint8_t)p->fixed[i];
        else if (p->fixed[i] == 2) xi = p->c[i] < 0;
        else {
            double sum = 0.0;
            for (int64_t q = vs0[i]; q < vs0[i + 1]; ++q) sum += M[vsl[q]];
            xi = sum < 0; /* at agreement every M_ij < 0 iff the sum is */
        }
        x[i] = xi;
        obj += p->c[i] * xi;
    }
    free(m0); free(m1); free(M); free(vs0); free(vsl); free(fill);
    if (rounds_out) *rounds_out = round;
    if (obj_out) *obj_out = obj;
    if (margin_out) *margin_out = margin;
    return rc;
}

/* ------------------------------------------------------------------------- */
/* accessors for tests                                                        */
/* ------------------------------------------------------------------------- */
int orc_num_bdds(const orc_problem *p) { return p->m; }
int64_t orc_num_slots(const orc_problem *p) { return p->S; }
int64_t orc_num_nodes(const orc_problem *p) { return p->N; }
double orc_const_lb(const orc_problem *p) { return p->const_lb; }

/* per BDD: original row, number of layers, number of nodes, first slot */
int orc_bdd_info(const orc_problem *p, int j, int *row, int *k, int *nn, int64_t *slot0) {
    if (j < 0 || j >= p->m) return ORC_EINVAL;
    *row = p->row[j];
    *k = p->bdd[j].k;
    *nn = p->bdd[j].nn;
    *slot0 = p->slot0[j];
    return ORC_OK;
}

/* node structure of BDD j: lstart (k+1), lo and hi (nn) with TOP = -1, BOT = -2 */
int orc_bdd_nodes(const orc_problem *p, int j, int *lstart, int *lo, int *hi) {
    if (j < 0 || j >= p->m) return ORC_EINVAL;
    const bdd_t *b = &p->bdd[j];
    memcpy(lstart, b->lstart, sizeof(int) * (b->k + 1));
    memcpy(lo, b->lo, sizeof(int) * b->nn);
    memcpy(hi, b->hi, sizeof(int) * b->nn);
    return ORC_OK;
}

int orc_slot_vars(const orc_problem *p, int *var) {
    memcpy(var, p->svar, sizeof(int) * p->S);
    return ORC_OK;
}

/* fixed: -1 in a BDD, 0/1 fixed by presolve, 2 in no row */
int orc_fixed(const orc_problem *p, int8_t *fixed) {
    memcpy(fixed, p->fixed, p->n);
    return ORC_OK;
}

int orc_get_state(const orc_problem *p, double *hi, double *lo, double *db0, double *db1) {
    if (hi) memcpy(hi, p->hi, sizeof(double) * p->S);
    if (lo) memcpy(lo, p->lo, sizeof(double) * p->S);
    if (db0) memcpy(db0, p->Db0, sizeof(double) * p->n);
    if (db1) memcpy(db1, p->Db1, sizeof(double) * p->n);
    return ORC_OK;
}

/* set the plain multipliers lambda (hi = lambda, lo = 0) and, optionally, the
   deferred per-variable sums; used to evaluate another implementation's state */
int orc_set_state(orc_problem *p, const double *lambda, const double *db0, const double *db1) {
    for (int64_t s = 0; s < p->S; ++s) { p->hi[s] = lambda[s]; p->lo[s] = 0.0; }
    for (int i = 0; i < p->n; ++i) {
        p->Db0[i] = db0 ? db0[i] : 0.0;
        p->Db1[i] = db1 ? db1[i] : 0.0;
    }
    p->spb_valid = p->spf_valid = 0;
    return ORC_OK;
}

/* shortest-path labels of BDD j at lambda = hi - lo: SP(r, v) and SP(v, TOP) (Fig. 3) */
int orc_bdd_shortest_paths(const orc_problem *p, int j, double *f, double *g) {
    if (j < 0 || j >= p->m) return ORC_EINVAL;
    const bdd_t *b = &p->bdd[j];
    int64_t s0 = p->slot0[j];
    double *w0 = calloc(b->k, sizeof(double)), *w1 = malloc(sizeof(double) * b->k);
    for (int t = 0; t < b->k; ++t) w1[t] = p->hi[s0 + t] - p->lo[s0 + t];
    sp_forward(b, w0, w1, f);
    sp_backward(b, w0, w1, g);
    free(w0); free(w1);
    return ORC_OK;
}

/* plain objective c^T x for a given x */
double orc_objective(const orc_problem *p, const uint8_t *x) {
    double obj = 0.0;
    for (int i = 0; i < p->n; ++i) obj += p->c[i] * x[i];
    return obj;
}
