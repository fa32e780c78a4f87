/*
 * fbp_oracle.c -- plain, sequential, double-precision belief propagation with
 * local structure, written from the FastLBP paper (arXiv 2509.22337).
 *
 * TEST INFRASTRUCTURE.  This file is the checker the CUDA path is compared
 * against.  Only the test suite, the package smoke check and the benchmark's
 * CPU-baseline leg load the library built from it.  It shares no code, header,
 * table or constant generator with the CUDA library; the factor type codes and
 * strategy codes below are the input format, declared here independently.
 *
 * What each part follows:
 *   - factor graph and messages ............ Sec. 3.1-3.2, Eq. (1)-(3)
 *   - local-structure term lists ........... Sec. 3.3, Eq. (4); indicator
 *                                             array of Sec. 4.3.2
 *   - one message from a term list ......... Algorithm 1
 *   - edge dependency neighbourhood ........ Definition 1
 *   - update-strategy semantics ............ Definition 2 with Eq. (5)
 *   - dependency analysis (levels) ......... Algorithm 2 (Sec. 4.2.3)
 *   - two-phase level execution ............ Sec. 4.3.1
 *   - strategies PARALL/SEQFIX/TOPO ........ Table 1
 * Readings where the paper is silent (initial messages, unary potentials,
 * the noisy factor semantics, the convergence measure, the forward/backward
 * and residual strategies, the zero-mass guard) are marked "reading:" below.
 *
 * Parity pins live in the test suite: dense-table Eq. (2) against the term
 * lists, brute-force exact marginals on trees, the worked example of Sec. 2.1
 * for Algorithm 2, and the invariants of Theorems 1 and 2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* factor type codes (input format); O_TERMS: a generic factor whose local
 * structure is given explicitly as an indicator array (Sec. 4.3.2) */
enum { O_AND = 0, O_OR = 1, O_NOT = 2, O_EQ = 3, O_NOISY_IMPLY = 4, O_NOISY_AND = 5, O_PRIOR = 6,
       O_TERMS = 7 };
/* strategy codes (input format) */
enum { S_PARALL = 0, S_SEQFIX = 1, S_TOPO = 2, S_TOPO_FB = 3, S_RESIDUAL = 4, S_CUSTOM = 5 };

#define WILD (-1)

/* ------------------------------------------------------------------------ */
/* Local-structure term lists (Eq. 4).                                       */
/*                                                                           */
/* A factor over b binary variables is a sum of l weighted terms; term t     */
/* fixes variable j to ind[j*lmax + t] in {0,1} or leaves it free (WILD).    */
/* Premises are variables 0..n-1 and the output y is variable n = b-1.       */
/* reading: the noisy types.  NOISY_AND(p): y holds only through the rule:  */
/* all premises true gives y=1 with weight p and y=0 with 1-p; any false     */
/* premise forces y=0.  NOISY_IMPLY(p): all premises true gives y=1 with p   */
/* and y=0 with 1-p; a false premise leaves y free (Sec. 2.2's Horn          */
/* constraint).  PRIOR(p) is a unary factor (y=1):p, (y=0):1-p.              */
/* Returns l, or -1 if the type/arity is not valid or lmax is too small.     */
/* ------------------------------------------------------------------------ */
int orc_terms(int type, int b, double p, int8_t *ind, double *w, int lmax)
{
    int n = b - 1, l = 0, t, j, k;
    if (b < 1) return -1;
#define NEED(x) do { if ((x) > lmax) return -1; } while (0)
#define SET(j_, t_, c_) (ind[(j_) * lmax + (t_)] = (int8_t)(c_))
    switch (type) {
    case O_AND:      /* (1..1, y=1):1 ; (x_<k=1, x_k=0, rest *, y=0):1 */
    case O_NOISY_AND:/* (1..1,y=1):p ; (1..1,y=0):1-p ; (x_<k=1, x_k=0, *, y=0):1 */
    case O_NOISY_IMPLY: /* as NOISY_AND but y free when a premise fails */
        if (b < 2) return -1;
        NEED(n + 2);
        for (t = 0; t < lmax; t++) for (j = 0; j < b; j++) SET(j, t, -2);
        /* all premises true */
        for (j = 0; j < n; j++) SET(j, l, 1);
        SET(n, l, 1);
        w[l++] = (type == O_AND) ? 1.0 : p;
        if (type != O_AND) {
            for (j = 0; j < n; j++) SET(j, l, 1);
            SET(n, l, 0);
            w[l++] = 1.0 - p;
        }
        /* first false premise at k */
        for (k = 0; k < n; k++) {
            for (j = 0; j < n; j++) SET(j, l, j < k ? 1 : (j == k ? 0 : WILD));
            SET(n, l, type == O_NOISY_IMPLY ? WILD : 0);
            w[l++] = 1.0;
        }
        return l;
    case O_OR:       /* (0..0, y=0):1 ; (x_<k=0, x_k=1, rest *, y=1):1 */
        if (b < 2) return -1;
        NEED(n + 1);
        for (t = 0; t < lmax; t++) for (j = 0; j < b; j++) SET(j, t, -2);
        for (j = 0; j < n; j++) SET(j, l, 0);
        SET(n, l, 0);
        w[l++] = 1.0;
        for (k = 0; k < n; k++) {
            for (j = 0; j < n; j++) SET(j, l, j < k ? 0 : (j == k ? 1 : WILD));
            SET(n, l, 1);
            w[l++] = 1.0;
        }
        return l;
    case O_NOT:      /* (x=0,y=1):1 ; (x=1,y=0):1 */
        if (b != 2) return -1;
        NEED(2);
        for (t = 0; t < lmax; t++) for (j = 0; j < b; j++) SET(j, t, -2);
        SET(0, 0, 0); SET(1, 0, 1); w[0] = 1.0;
        SET(0, 1, 1); SET(1, 1, 0); w[1] = 1.0;
        return 2;
    case O_EQ:       /* (all 0):1 ; (all 1):1 */
        NEED(2);
        for (t = 0; t < lmax; t++) for (j = 0; j < b; j++) SET(j, t, -2);
        for (j = 0; j < b; j++) { SET(j, 0, 0); SET(j, 1, 1); }
        w[0] = 1.0; w[1] = 1.0;
        return 2;
    case O_PRIOR:    /* (y=1):p ; (y=0):1-p */
        if (b != 1) return -1;
        NEED(2);
        SET(0, 0, 1); w[0] = p;
        SET(0, 1, 0); w[1] = 1.0 - p;
        return 2;
    default:
        return -1;
    }
#undef NEED
#undef SET
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: one factor-to-variable message entry mu_{a->v}(x_v) as the   */
/* sum of the sub-messages of the terms that do not conflict with x_v.       */
/* mu[j*2 + c] is the incoming message from variable j at value c (r = 2).   */
/* ------------------------------------------------------------------------ */
double orc_alg1(int b, int l, int lmax, const int8_t *ind, const double *w,
                const double *mu, int v, int xv)
{
    double message = 0.0;
    for (int t = 0; t < l; t++) {
        int iv = ind[v * lmax + t];
        if (iv != xv && iv != WILD) continue;      /* term conflicts with x_v */
        double sm = w[t];
        for (int j = 0; j < b; j++) {
            if (j == v) continue;
            int c = ind[j * lmax + t];
            if (c == WILD) sm *= mu[j * 2 + 0] + mu[j * 2 + 1];
            else           sm *= mu[j * 2 + c];
        }
        message += sm;
    }
    return message;
}

/* reading: the zero-mass guard.  A message whose two entries sum to zero
 * (contradictory hard evidence through deterministic factors) or to a
 * non-finite value is replaced by the uniform message; the guard is counted. */
static int normalize_guard(double m[2])
{
    double s = m[0] + m[1];
    if (!(s > 0.0) || !isfinite(s)) { m[0] = 0.5; m[1] = 0.5; return 1; }
    m[0] /= s; m[1] /= s;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Graph                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t nv, na;
    int64_t ne;
    int64_t *fptr;      /* [na+1] factor-major CSR (edge id = position) */
    int32_t *fvars;     /* [ne] */
    uint8_t *ftype;     /* [na] */
    double *fparam;     /* [na] */
    int32_t *efac;      /* [ne] factor of each edge */
    int64_t *vptr;      /* [nv+1] variable-major adjacency */
    int64_t *vedge;     /* [ne] edge ids of each variable, ascending */
    double *phi;        /* [2*nv] unary potential of each variable */
    /* per-factor term lists */
    int *nterms; int lmax; int8_t **ind; double **tw;
} og_graph;

void orc_graph_free(og_graph *g)
{
    if (!g) return;
    if (g->ind) for (int a = 0; a < g->na; a++) { free(g->ind[a]); free(g->tw[a]); }
    free(g->ind); free(g->tw); free(g->nterms);
    free(g->fptr); free(g->fvars); free(g->ftype); free(g->fparam); free(g->efac);
    free(g->vptr); free(g->vedge); free(g->phi);
    free(g);
}

/* reading: unary potentials.  Evidence x=0 gives phi=(1,0), x=1 gives (0,1);
 * otherwise a prior p gives (1-p,p); otherwise (1,1).  phi multiplies into
 * Eq. (1) and Eq. (3) like an extra incoming message. */
static void set_phi(og_graph *g, int32_t v, float prior, int8_t ev)
{
    double *f = g->phi + 2 * (int64_t)v;
    if (ev == 0)      { f[0] = 1.0; f[1] = 0.0; }
    else if (ev == 1) { f[0] = 0.0; f[1] = 1.0; }
    else if (!isnan(prior)) { f[0] = 1.0 - (double)prior; f[1] = (double)prior; }
    else              { f[0] = 1.0; f[1] = 1.0; }
}

og_graph *orc_graph_new(int32_t nv, int32_t na, const int64_t *fptr, const int32_t *fvars,
                        const uint8_t *ftype, const float *fparam, const float *prior,
                        const int8_t *evidence)
{
    if (nv < 0 || na < 0) return NULL;
    og_graph *g = (og_graph *)calloc(1, sizeof(og_graph));
    g->nv = nv; g->na = na; g->ne = fptr[na];
    g->fptr = (int64_t *)malloc(sizeof(int64_t) * (na + 1));
    g->fvars = (int32_t *)malloc(sizeof(int32_t) * (g->ne + 1));
    g->ftype = (uint8_t *)malloc(na + 1);
    g->fparam = (double *)malloc(sizeof(double) * (na + 1));
    g->efac = (int32_t *)malloc(sizeof(int32_t) * (g->ne + 1));
    g->vptr = (int64_t *)calloc(nv + 1, sizeof(int64_t));
    g->vedge = (int64_t *)malloc(sizeof(int64_t) * (g->ne + 1));
    g->phi = (double *)malloc(sizeof(double) * 2 * (nv + 1));
    memcpy(g->fptr, fptr, sizeof(int64_t) * (na + 1));
    memcpy(g->fvars, fvars, sizeof(int32_t) * g->ne);
    memcpy(g->ftype, ftype, na);
    for (int a = 0; a < na; a++) g->fparam[a] = (double)fparam[a];
    if (fptr[0] != 0) { orc_graph_free(g); return NULL; }
    for (int a = 0; a < na; a++) {
        if (fptr[a + 1] < fptr[a]) { orc_graph_free(g); return NULL; }
        for (int64_t e = fptr[a]; e < fptr[a + 1]; e++) {
            if (fvars[e] < 0 || fvars[e] >= nv) { orc_graph_free(g); return NULL; }
            for (int64_t q = fptr[a]; q < e; q++)   /* a variable appears once per factor */
                if (fvars[q] == fvars[e]) { orc_graph_free(g); return NULL; }
            g->efac[e] = a;
            g->vptr[fvars[e] + 1]++;
        }
    }
    if (evidence)
        for (int32_t v = 0; v < nv; v++)
            if (evidence[v] < -1 || evidence[v] > 1) { orc_graph_free(g); return NULL; }
    for (int32_t v = 0; v < nv; v++) g->vptr[v + 1] += g->vptr[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nv + 1));
    memcpy(fill, g->vptr, sizeof(int64_t) * (nv + 1));
    for (int64_t e = 0; e < g->ne; e++) g->vedge[fill[fvars[e]]++] = e;
    free(fill);
    for (int32_t v = 0; v < nv; v++)
        set_phi(g, v, prior ? prior[v] : NAN, evidence ? evidence[v] : (int8_t)-1);
    /* term lists, one per factor */
    int lmax = 2;
    for (int a = 0; a < na; a++) {
        int b = (int)(fptr[a + 1] - fptr[a]);
        if (b + 1 > lmax) lmax = b + 1;
    }
    g->lmax = lmax;
    g->nterms = (int *)malloc(sizeof(int) * (na + 1));
    g->ind = (int8_t **)calloc(na + 1, sizeof(int8_t *));
    g->tw = (double **)calloc(na + 1, sizeof(double *));
    for (int a = 0; a < na; a++) {
        int b = (int)(fptr[a + 1] - fptr[a]);
        g->ind[a] = (int8_t *)malloc((size_t)(b > 0 ? b : 1) * lmax);
        g->tw[a] = (double *)malloc(sizeof(double) * lmax);
        if (ftype[a] == O_TERMS) {  /* terms come from orc_set_terms */
            if (b < 1) { orc_graph_free(g); return NULL; }
            g->nterms[a] = 0;
            continue;
        }
        g->nterms[a] = orc_terms(ftype[a], b, g->fparam[a], g->ind[a], g->tw[a], lmax);
        if (g->nterms[a] < 0) { orc_graph_free(g); return NULL; }
    }
    return g;
}

/* ------------------------------------------------------------------------ */
/* Explicit local structure of the generic (O_TERMS) factors: the indicator   */
/* array of Sec. 4.3.2 and its weights, evaluated by Algorithm 1 like every   */
/* other factor.  Factor a's terms are term_ptr[a] .. term_ptr[a+1]-1; its    */
/* indicators are a block of (terms x variables) values, term after term, in  */
/* the factor's variable order, blocks in factor order; a value is 0, 1 or    */
/* -1 (the variable is free in that term).  Other factors must have no terms. */
/* The term store is re-laid with a larger common stride when needed.         */
/* ------------------------------------------------------------------------ */
int orc_set_terms(og_graph *g, const int64_t *term_ptr, const int8_t *term_ind, const double *term_w)
{
    int need = g->lmax;
    if (term_ptr[0] != 0) return -1;
    for (int a = 0; a < g->na; a++) {
        int64_t l = term_ptr[a + 1] - term_ptr[a];
        if (l < 0 || (g->ftype[a] != O_TERMS && l != 0)) return -1;
        if (l > need) need = (int)l;
    }
    int64_t off = 0;
    for (int a = 0; a < g->na; a++) {
        int b = (int)(g->fptr[a + 1] - g->fptr[a]);
        for (int64_t t = term_ptr[a]; t < term_ptr[a + 1]; t++) {
            if (!(term_w[t] >= 0.0) || !isfinite(term_w[t])) return -1;
            for (int j = 0; j < b; j++) {
                int8_t c = term_ind[off + (t - term_ptr[a]) * b + j];
                if (c < -1 || c > 1) return -1;
            }
        }
        off += (term_ptr[a + 1] - term_ptr[a]) * b;
    }
    if (need > g->lmax) {  /* re-lay every factor's terms with the new stride */
        for (int a = 0; a < g->na; a++) {
            int b = (int)(g->fptr[a + 1] - g->fptr[a]);
            int8_t *ind = (int8_t *)malloc((size_t)(b > 0 ? b : 1) * need);
            double *tw = (double *)malloc(sizeof(double) * need);
            for (int j = 0; j < b; j++)
                for (int t = 0; t < g->nterms[a]; t++) ind[j * need + t] = g->ind[a][j * g->lmax + t];
            for (int t = 0; t < g->nterms[a]; t++) tw[t] = g->tw[a][t];
            free(g->ind[a]); free(g->tw[a]);
            g->ind[a] = ind; g->tw[a] = tw;
        }
        g->lmax = need;
    }
    off = 0;
    for (int a = 0; a < g->na; a++) {
        int b = (int)(g->fptr[a + 1] - g->fptr[a]);
        int l = (int)(term_ptr[a + 1] - term_ptr[a]);
        if (g->ftype[a] == O_TERMS) {
            for (int t = 0; t < l; t++) {
                for (int j = 0; j < b; j++) {
                    int8_t c = term_ind[off + (int64_t)t * b + j];
                    g->ind[a][j * g->lmax + t] = (int8_t)(c < 0 ? WILD : c);
                }
                g->tw[a][t] = term_w[term_ptr[a] + t];
            }
            g->nterms[a] = l;
        }
        off += (int64_t)l * b;
    }
    return 0;
}

int64_t orc_num_edges(const og_graph *g) { return g->ne; }

int orc_set_evidence(og_graph *g, int32_t v, int8_t value, float prior)
{
    if (v < 0 || v >= g->nv) return -1;
    set_phi(g, v, prior, value);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. (1): variable-to-factor messages.                                     */
/* ------------------------------------------------------------------------ */
#define TINY 0x1p-500
#define HUGE_ 0x1p500

static void rescale(double m[2])
{
    double mx = m[0] > m[1] ? m[0] : m[1];
    if (mx > 0.0 && mx < TINY) { m[0] *= HUGE_; m[1] *= HUGE_; }
}

/* mu_{v->a} for the edge e_out = (a, v): phi_v times the product of every
 * incoming factor-to-variable message of v except the one on e_out, taken
 * literally; the pair is rescaled by a power of two whenever it gets tiny
 * (this leaves the normalised message unchanged), then normalised. */
static int v2a_literal(const og_graph *g, const double *a2v, int32_t v, int64_t e_out, double out[2])
{
    double m[2] = { g->phi[2 * v], g->phi[2 * v + 1] };
    for (int64_t k = g->vptr[v]; k < g->vptr[v + 1]; k++) {
        int64_t e = g->vedge[k];
        if (e == e_out) continue;
        m[0] *= a2v[2 * e];
        m[1] *= a2v[2 * e + 1];
        rescale(m);
    }
    out[0] = m[0]; out[1] = m[1];
    return normalize_guard(out);
}

/* All mu_{v->a} of variable v's row at once: for rows longer than 64 the
 * exclusion product is a prefix product times a suffix product (the same
 * product as above, grouped differently) so that a hub costs O(degree). */
static int64_t v2a_row(const og_graph *g, const double *a2v, int32_t v, double *v2a,
                       double *scratch)
{
    int64_t d = g->vptr[v + 1] - g->vptr[v], guards = 0;
    const int64_t *row = g->vedge + g->vptr[v];
    if (d <= 64) {
        for (int64_t k = 0; k < d; k++) guards += v2a_literal(g, a2v, v, row[k], v2a + 2 * row[k]);
        return guards;
    }
    double *pre = scratch, *suf = scratch + 2 * (d + 1);
    pre[0] = 1.0; pre[1] = 1.0;
    for (int64_t k = 0; k < d; k++) {
        double m[2] = { pre[2 * k] * a2v[2 * row[k]], pre[2 * k + 1] * a2v[2 * row[k] + 1] };
        rescale(m);
        pre[2 * (k + 1)] = m[0]; pre[2 * (k + 1) + 1] = m[1];
    }
    suf[2 * d] = 1.0; suf[2 * d + 1] = 1.0;
    for (int64_t k = d - 1; k >= 0; k--) {
        double m[2] = { suf[2 * (k + 1)] * a2v[2 * row[k]], suf[2 * (k + 1) + 1] * a2v[2 * row[k] + 1] };
        rescale(m);
        suf[2 * k] = m[0]; suf[2 * k + 1] = m[1];
    }
    for (int64_t k = 0; k < d; k++) {
        double m[2] = { pre[2 * k] * suf[2 * (k + 1)], pre[2 * k + 1] * suf[2 * (k + 1) + 1] };
        rescale(m);
        m[0] *= g->phi[2 * v]; m[1] *= g->phi[2 * v + 1];
        guards += normalize_guard(m);
        v2a[2 * row[k]] = m[0]; v2a[2 * row[k] + 1] = m[1];
    }
    return guards;
}

/* Exposed for the tests: the v->a messages of one variable's row, computed
 * both literally and through v2a_row (prefix/suffix for long rows). */
int orc_v2a_row(const og_graph *g, const double *a2v, int32_t v, double *v2a_all, int literal)
{
    int64_t d = g->vptr[v + 1] - g->vptr[v];
    if (literal) {
        for (int64_t k = g->vptr[v]; k < g->vptr[v + 1]; k++)
            v2a_literal(g, a2v, v, g->vedge[k], v2a_all + 2 * g->vedge[k]);
        return 0;
    }
    double *scr = (double *)malloc(sizeof(double) * 4 * (d + 2));
    v2a_row(g, a2v, v, v2a_all, scr);
    free(scr);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Phase 2 for one edge: mu_{a->v} by Algorithm 1 over the factor's term     */
/* list, from the v->a messages of the factor's row; normalised with guard.  */
/* ------------------------------------------------------------------------ */
static int a2v_alg1(const og_graph *g, const double *v2a, int64_t e, double out[2], double *mu)
{
    int32_t a = g->efac[e];
    int b = (int)(g->fptr[a + 1] - g->fptr[a]);
    int pos = (int)(e - g->fptr[a]);
    for (int j = 0; j < b; j++) {
        mu[2 * j] = v2a[2 * (g->fptr[a] + j)];
        mu[2 * j + 1] = v2a[2 * (g->fptr[a] + j) + 1];
    }
    out[0] = orc_alg1(b, g->nterms[a], g->lmax, g->ind[a], g->tw[a], mu, pos, 0);
    out[1] = orc_alg1(b, g->nterms[a], g->lmax, g->ind[a], g->tw[a], mu, pos, 1);
    return normalize_guard(out);
}

/* ------------------------------------------------------------------------ */
/* Update strategy -> integer rank per edge (a weak order; Table 1).         */
/*   PARALL: every edge in one class.                                        */
/*   SEQFIX: a total order; rank = given order or the edge id.               */
/*   TOPO: reading: rank(a,v) = depth of the output (last) variable of a,    */
/*     depth(u) = 0 without a defining factor, else the largest             */
/*     1 + max premise depth over the factors whose output is u (an empty    */
/*     premise list counts as depth -1).  Cyclic graphs are rejected (-4).   */
/*   backward: rank -> (max rank - rank), for the backward half of TOPO_FB.  */
/* ------------------------------------------------------------------------ */
int orc_ranks(const og_graph *g, int strategy, const int64_t *custom, int backward, int64_t *rank)
{
    int64_t E = g->ne;
    if (strategy == S_PARALL) {
        for (int64_t e = 0; e < E; e++) rank[e] = 0;
    } else if (strategy == S_SEQFIX || strategy == S_CUSTOM) {
        if (strategy == S_CUSTOM && !custom) return -1;
        for (int64_t e = 0; e < E; e++) rank[e] = custom ? custom[e] : e;
    } else if (strategy == S_TOPO || strategy == S_TOPO_FB) {
        int32_t nv = g->nv, na = g->na;
        /* Kahn's algorithm over variables: premise -> output of every factor */
        int64_t *indeg = (int64_t *)calloc(nv + 1, sizeof(int64_t));
        int64_t *depth = (int64_t *)calloc(nv + 1, sizeof(int64_t));
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (nv + 1));
        /* out-lists: for each variable, the factors in which it is a premise */
        int64_t *optr = (int64_t *)calloc(nv + 1, sizeof(int64_t));
        int32_t *ofac;
        for (int32_t a = 0; a < na; a++) {
            int64_t lo = g->fptr[a], hi = g->fptr[a + 1];
            if (hi - lo < 1) continue;
            indeg[g->fvars[hi - 1]] += hi - 1 - lo;
            for (int64_t e = lo; e < hi - 1; e++) optr[g->fvars[e] + 1]++;
        }
        for (int32_t v = 0; v < nv; v++) optr[v + 1] += optr[v];
        ofac = (int32_t *)malloc(sizeof(int32_t) * (optr[nv] + 1));
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nv + 1));
        memcpy(fill, optr, sizeof(int64_t) * (nv + 1));
        for (int32_t a = 0; a < na; a++) {
            int64_t lo = g->fptr[a], hi = g->fptr[a + 1];
            for (int64_t e = lo; e < hi - 1; e++) ofac[fill[g->fvars[e]]++] = a;
        }
        free(fill);
        /* a variable defined by a factor with no premises has depth 0 */
        int32_t qh = 0, qt = 0;
        for (int32_t v = 0; v < nv; v++) if (indeg[v] == 0) queue[qt++] = v;
        while (qh < qt) {
            int32_t u = queue[qh++];
            for (int64_t k = optr[u]; k < optr[u + 1]; k++) {
                int32_t a = ofac[k];
                int32_t y = g->fvars[g->fptr[a + 1] - 1];
                if (depth[u] + 1 > depth[y]) depth[y] = depth[u] + 1;
                if (--indeg[y] == 0) queue[qt++] = y;
            }
        }
        int cyclic = qt < nv;
        if (!cyclic) {
            int64_t mx = 0;
            for (int32_t a = 0; a < na; a++)
                for (int64_t e = g->fptr[a]; e < g->fptr[a + 1]; e++) {
                    rank[e] = depth[g->fvars[g->fptr[a + 1] - 1]];
                    if (rank[e] > mx) mx = rank[e];
                }
            if (backward) for (int64_t e = 0; e < E; e++) rank[e] = mx - rank[e];
        }
        free(indeg); free(depth); free(queue); free(optr); free(ofac);
        return cyclic ? -4 : 0;
    } else {
        return -1;
    }
    if (backward) {
        int64_t mx = 0;
        for (int64_t e = 0; e < E; e++) if (rank[e] > mx) mx = rank[e];
        for (int64_t e = 0; e < E; e++) rank[e] = mx - rank[e];
    }
    return 0;
}

/* canonical order: edges sorted by (rank, edge id) -- the topological sort of
 * Algorithm 2 with edges of one equivalence class kept in edge-id order */
static const int64_t *g_sort_rank;
static int cmp_rank(const void *x, const void *y)
{
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    if (g_sort_rank[a] != g_sort_rank[b]) return g_sort_rank[a] < g_sort_rank[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

static int64_t *canonical_order(const int64_t *rank, const int64_t *edges, int64_t n)
{
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    memcpy(ord, edges, sizeof(int64_t) * n);
    g_sort_rank = rank;
    qsort(ord, n, sizeof(int64_t), cmp_rank);
    return ord;
}

/* Definition 1: is e in N_E(f)?  N_E((a,v)) holds the edges (a*,v*) with v*
 * a neighbour of a other than v and a* a neighbour of v* other than a. */
int orc_in_ne(const og_graph *g, int64_t e, int64_t f)
{
    int32_t a = g->efac[f], v = g->fvars[f];
    int32_t as = g->efac[e], vs = g->fvars[e];
    if (as == a || vs == v) return 0;
    for (int64_t k = g->fptr[a]; k < g->fptr[a + 1]; k++)
        if (g->fvars[k] == vs) return 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, literally: scan the edges in canonical order; before adding  */
/* e_i, look through NextSet for an edge e with e in N_E(e_i) and e < e_i    */
/* (strictly earlier class); if one exists, close NextSet as a level.        */
/* `edges` restricts the analysis to a subset (all edges when NULL).         */
/* Writes level_ptr[k+1] and level_edges[n]; returns k.                      */
/* ------------------------------------------------------------------------ */
int64_t orc_levels_literal(const og_graph *g, const int64_t *rank, const int64_t *edges, int64_t n,
                           int64_t *level_ptr, int32_t *level_edges)
{
    int64_t *all = NULL;
    if (!edges) {
        n = g->ne;
        all = (int64_t *)calloc(n + 1, sizeof(int64_t));
        for (int64_t e = 0; e < n; e++) all[e] = e;
        edges = all;
    }
    int64_t *ord = canonical_order(rank, edges, n);
    int64_t k = 0, next_lo = 0;   /* NextSet = ord[next_lo .. i) */
    level_ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t ei = ord[i];
        for (int64_t j = next_lo; j < i; j++) {
            int64_t e = ord[j];
            if (rank[e] < rank[ei] && orc_in_ne(g, e, ei)) {
                level_ptr[++k] = i;   /* S.append(NextSet) */
                next_lo = i;
                break;
            }
        }
        level_edges[i] = (int32_t)ei;   /* NextSet <- NextSet + {e_i} */
    }
    if (n > 0) level_ptr[++k] = n;
    free(ord); free(all);
    return k;
}

/* Algorithm 2 with the inner scan turned around: instead of walking NextSet
 * and testing membership in N_E(e_i), walk N_E(e_i) (Definition 1) and test
 * membership in NextSet.  Same predicate, same output; used where the literal
 * scan is too slow, and checked against it in the tests. */
int64_t orc_levels_nbr(const og_graph *g, const int64_t *rank, const int64_t *edges, int64_t n,
                       int64_t *level_ptr, int32_t *level_edges)
{
    int64_t *all = NULL;
    if (!edges) {
        n = g->ne;
        all = (int64_t *)calloc(n + 1, sizeof(int64_t));
        for (int64_t e = 0; e < n; e++) all[e] = e;
        edges = all;
    }
    int64_t *ord = canonical_order(rank, edges, n);
    int64_t *in_level = (int64_t *)malloc(sizeof(int64_t) * (g->ne + 1));
    for (int64_t e = 0; e < g->ne; e++) in_level[e] = -1;
    int64_t k = 0;
    level_ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t ei = ord[i];
        int32_t a = g->efac[ei], v = g->fvars[ei];
        int cut = 0;
        for (int64_t q = g->fptr[a]; q < g->fptr[a + 1] && !cut; q++) {
            int32_t vs = g->fvars[q];
            if (vs == v) continue;
            for (int64_t r = g->vptr[vs]; r < g->vptr[vs + 1]; r++) {
                int64_t e = g->vedge[r];
                if (g->efac[e] == a) continue;
                if (in_level[e] == k && rank[e] < rank[ei]) { cut = 1; break; }
            }
        }
        if (cut) level_ptr[++k] = i;
        in_level[ei] = k;
        level_edges[i] = (int32_t)ei;
    }
    if (n > 0) level_ptr[++k] = n;
    free(ord); free(all); free(in_level);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Level-mode execution (Sec. 4.3.1): for each level, phase 1 computes the   */
/* v->a messages of every variable adjacent to a factor the level touches,   */
/* from the messages as they stand at the start of the level; phase 2        */
/* computes the level's a->v messages from those (Algorithm 1); then the new */
/* messages are stored.  Tracks the largest |new m1 - old m1| (reading: the  */
/* convergence measure) and the count of zero-mass guards.                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    double *v2a, *newm, *scratch, *mu;
    int64_t *fstamp, *vstamp, stamp;
    double *dres;   /* optional: per-edge |delta m1| of the last write */
    double min_pos; /* diagnostic: smallest nonzero entry of any written message */
} run_ws;

static void note_min(run_ws *ws, const double *m)
{
    if (m[0] > 0.0 && m[0] < ws->min_pos) ws->min_pos = m[0];
    if (m[1] > 0.0 && m[1] < ws->min_pos) ws->min_pos = m[1];
}

/* Host threads a run may use (orc_set_threads).  With more than one, each
 * level's phase 1 runs over the level's distinct variables in parallel, and
 * phase 2 and the store over the level's edges in parallel: every one of
 * those updates reads only the level-start messages and writes its own
 * entries, and the residual, guard count and range diagnostic are a max, a
 * sum and a min, so the results are the same as with one thread.  This is
 * for timing the oracle on every host core; the arithmetic is unchanged. */
static int g_threads = 1;

int orc_set_threads(int n)
{
#ifdef _OPENMP
    int mx = omp_get_num_procs();
    g_threads = n < 1 ? 1 : n > mx ? mx : n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

static void run_levels(const og_graph *g, double *a2v, int64_t k, const int64_t *level_ptr,
                       const int32_t *level_edges, run_ws *ws, double *residual, int64_t *guards);

#ifdef _OPENMP
static void run_levels_threads(const og_graph *g, double *a2v, int64_t k, const int64_t *level_ptr,
                               const int32_t *level_edges, run_ws *ws, double *residual, int64_t *guards)
{
    int64_t maxd = 1;
    for (int32_t v = 0; v < g->nv; v++)
        if (g->vptr[v + 1] - g->vptr[v] > maxd) maxd = g->vptr[v + 1] - g->vptr[v];
    int bmax = 1;
    for (int32_t a = 0; a < g->na; a++)
        if (g->fptr[a + 1] - g->fptr[a] > bmax) bmax = (int)(g->fptr[a + 1] - g->fptr[a]);
    const int T = g_threads;
    double *scratch = (double *)malloc(sizeof(double) * 4 * (maxd + 2) * T);
    double *mu = (double *)malloc(sizeof(double) * 2 * (bmax + 1) * T);
    int32_t *vars = (int32_t *)malloc(sizeof(int32_t) * (g->nv + 1));
    for (int64_t L = 0; L < k; L++) {
        int64_t lo = level_ptr[L], hi = level_ptr[L + 1], nvl = 0;
        ws->stamp++;
        for (int64_t i = lo; i < hi; i++) {
            int32_t a = g->efac[level_edges[i]];
            if (ws->fstamp[a] == ws->stamp) continue;
            ws->fstamp[a] = ws->stamp;
            for (int64_t q = g->fptr[a]; q < g->fptr[a + 1]; q++) {
                int32_t v = g->fvars[q];
                if (ws->vstamp[v] == ws->stamp) continue;
                ws->vstamp[v] = ws->stamp;
                vars[nvl++] = v;
            }
        }
#pragma omp parallel for num_threads(T) schedule(dynamic, 256)
        for (int64_t j = 0; j < nvl; j++)
            v2a_row(g, a2v, vars[j], ws->v2a, scratch + 4 * (maxd + 2) * omp_get_thread_num());
        int64_t gsum = 0;
#pragma omp parallel for num_threads(T) schedule(dynamic, 1024) reduction(+ : gsum)
        for (int64_t i = lo; i < hi; i++)
            gsum += a2v_alg1(g, ws->v2a, level_edges[i], ws->newm + 2 * (i - lo),
                             mu + 2 * (bmax + 1) * omp_get_thread_num());
        *guards += gsum;
        double res = *residual, mp = ws->min_pos;
#pragma omp parallel for num_threads(T) schedule(static) reduction(max : res) reduction(min : mp)
        for (int64_t i = lo; i < hi; i++) {
            int64_t e = level_edges[i];
            const double *nm = ws->newm + 2 * (i - lo);
            double d = fabs(nm[1] - a2v[2 * e + 1]);
            if (d > res) res = d;
            if (ws->dres) ws->dres[e] = d;
            if (nm[0] > 0.0 && nm[0] < mp) mp = nm[0];
            if (nm[1] > 0.0 && nm[1] < mp) mp = nm[1];
            a2v[2 * e] = nm[0];
            a2v[2 * e + 1] = nm[1];
        }
        *residual = res;
        ws->min_pos = mp;
    }
    free(scratch); free(mu); free(vars);
}
#endif

static void run_levels(const og_graph *g, double *a2v, int64_t k, const int64_t *level_ptr,
                       const int32_t *level_edges, run_ws *ws, double *residual, int64_t *guards)
{
#ifdef _OPENMP
    if (g_threads > 1) {
        run_levels_threads(g, a2v, k, level_ptr, level_edges, ws, residual, guards);
        return;
    }
#endif
    for (int64_t L = 0; L < k; L++) {
        int64_t lo = level_ptr[L], hi = level_ptr[L + 1];
        ws->stamp++;
        /* phase 1 */
        for (int64_t i = lo; i < hi; i++) {
            int32_t a = g->efac[level_edges[i]];
            if (ws->fstamp[a] == ws->stamp) continue;
            ws->fstamp[a] = ws->stamp;
            for (int64_t q = g->fptr[a]; q < g->fptr[a + 1]; q++) {
                int32_t v = g->fvars[q];
                if (ws->vstamp[v] == ws->stamp) continue;
                ws->vstamp[v] = ws->stamp;
                v2a_row(g, a2v, v, ws->v2a, ws->scratch);
            }
        }
        /* phase 2 */
        for (int64_t i = lo; i < hi; i++) {
            int64_t e = level_edges[i];
            *guards += a2v_alg1(g, ws->v2a, e, ws->newm + 2 * (i - lo), ws->mu);
        }
        /* store */
        for (int64_t i = lo; i < hi; i++) {
            int64_t e = level_edges[i];
            double d = fabs(ws->newm[2 * (i - lo) + 1] - a2v[2 * e + 1]);
            if (d > *residual) *residual = d;
            if (ws->dres) ws->dres[e] = d;
            note_min(ws, ws->newm + 2 * (i - lo));
            a2v[2 * e] = ws->newm[2 * (i - lo)];
            a2v[2 * e + 1] = ws->newm[2 * (i - lo) + 1];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Definition-2 execution: walk the edges in canonical order; for every      */
/* dependency e' in N_E(e) take the current-iteration value when e' is in a  */
/* strictly earlier class than e (delta = 1) and the previous iteration's    */
/* value otherwise (Eq. 5).                                                  */
/* ------------------------------------------------------------------------ */
static void run_def2(const og_graph *g, double *a2v, const int64_t *rank, const int64_t *ord,
                     double *oldm, run_ws *ws, double *residual, int64_t *guards)
{
    memcpy(oldm, a2v, sizeof(double) * 2 * g->ne);
    for (int64_t i = 0; i < g->ne; i++) {
        int64_t e = ord[i];
        int32_t a = g->efac[e];
        int b = (int)(g->fptr[a + 1] - g->fptr[a]);
        for (int j = 0; j < b; j++) {
            int64_t q = g->fptr[a] + j;
            int32_t vs = g->fvars[q];
            double m[2] = { g->phi[2 * vs], g->phi[2 * vs + 1] };
            for (int64_t r = g->vptr[vs]; r < g->vptr[vs + 1]; r++) {
                int64_t ep = g->vedge[r];
                if (ep == q) continue;          /* a* != a */
                const double *src = rank[ep] < rank[e] ? a2v : oldm;
                m[0] *= src[2 * ep]; m[1] *= src[2 * ep + 1];
                rescale(m);
            }
            normalize_guard(m);
            ws->v2a[2 * q] = m[0]; ws->v2a[2 * q + 1] = m[1];
        }
        double out[2];
        *guards += a2v_alg1(g, ws->v2a, e, out, ws->mu);
        double d = fabs(out[1] - oldm[2 * e + 1]);
        if (d > *residual) *residual = d;
        note_min(ws, out);
        a2v[2 * e] = out[0]; a2v[2 * e + 1] = out[1];
    }
}

/* ------------------------------------------------------------------------ */
/* reading: the residual strategy (cited in Sec. 1 but not expressed in the  */
/* IR).  Iteration 1 updates every edge in one class.  For iteration t >= 2  */
/* factor a gets priority rho_a = the largest |delta m1| of the iteration-   */
/* (t-1) writes into any variable of a; factors with rho_a >= 1e-2 form      */
/* class 0, [1e-4, 1e-2) class 1, [tol, 1e-4) class 2, and factors below     */
/* tol are skipped.  Algorithm 2 runs on the active edges with those ranks.  */
/* ------------------------------------------------------------------------ */
static int64_t residual_active(const og_graph *g, const double *dres, double tol, int64_t *rank,
                               int64_t *edges, double *vres)
{
    int64_t n = 0;
    for (int32_t v = 0; v < g->nv; v++) {
        double r = 0.0;
        for (int64_t k = g->vptr[v]; k < g->vptr[v + 1]; k++)
            if (dres[g->vedge[k]] > r) r = dres[g->vedge[k]];
        vres[v] = r;
    }
    for (int32_t a = 0; a < g->na; a++) {
        double rho = 0.0;
        for (int64_t q = g->fptr[a]; q < g->fptr[a + 1]; q++)
            if (vres[g->fvars[q]] > rho) rho = vres[g->fvars[q]];
        int64_t cls = rho >= 1e-2 ? 0 : rho >= 1e-4 ? 1 : rho >= tol ? 2 : -1;
        for (int64_t q = g->fptr[a]; q < g->fptr[a + 1]; q++) {
            rank[q] = cls;
            if (cls >= 0) edges[n++] = q;
        }
    }
    return n;
}

/* Exposed for the tests: the residual strategy's class of every edge (rank,
 * -1 = skipped) and its active edges, from given previous-iteration per-edge
 * |delta m1| values.  Returns the number of active edges. */
int64_t orc_residual_classes(const og_graph *g, const double *dres, double tol, int64_t *rank,
                             int64_t *edges)
{
    double *vres = (double *)malloc(sizeof(double) * (g->nv + 1));
    int64_t n = residual_active(g, dres, tol, rank, edges, vres);
    free(vres);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Full run.  a2v holds 2*E doubles: (m0, m1) per edge; if init is zero it   */
/* is set to the uniform message first (reading: initial messages).          */
/* Iteration t's residual is the largest |delta m1| over its writes; the run */
/* stops at the first t with residual < tol (returns 0, iters = t) or after  */
/* max_iters (returns 1).  TOPO_FB runs the forward then the backward        */
/* levels in one iteration.  def2 = 1 executes Definition 2 directly instead */
/* of the levels.  res_hist (optional) receives each iteration's residual;   */
/* updates_out (optional) the number of a->v writes; min_pos_out (optional)  */
/* the smallest nonzero entry of any message written (a range diagnostic:    */
/* it tells whether the run stayed within single-precision range).           */
/* ------------------------------------------------------------------------ */
int orc_run(og_graph *g, int strategy, const int64_t *custom, int max_iters, double tol,
            int def2, int init, double *a2v, int32_t *iters_out, double *residual_out,
            double *res_hist, int64_t *guards_out, int64_t *updates_out, double *min_pos_out)
{
    int64_t E = g->ne;
    int64_t maxd = 1;
    for (int32_t v = 0; v < g->nv; v++)
        if (g->vptr[v + 1] - g->vptr[v] > maxd) maxd = g->vptr[v + 1] - g->vptr[v];
    int bmax = 1;
    for (int32_t a = 0; a < g->na; a++)
        if (g->fptr[a + 1] - g->fptr[a] > bmax) bmax = (int)(g->fptr[a + 1] - g->fptr[a]);
    run_ws ws;
    memset(&ws, 0, sizeof(ws));
    ws.min_pos = 1.0;
    ws.v2a = (double *)malloc(sizeof(double) * 2 * (E + 1));
    ws.newm = (double *)malloc(sizeof(double) * 2 * (E + 1));
    ws.scratch = (double *)malloc(sizeof(double) * 4 * (maxd + 2));
    ws.mu = (double *)malloc(sizeof(double) * 2 * (bmax + 1));
    ws.fstamp = (int64_t *)calloc(g->na + 1, sizeof(int64_t));
    ws.vstamp = (int64_t *)calloc(g->nv + 1, sizeof(int64_t));
    int64_t *rank = (int64_t *)malloc(sizeof(int64_t) * (E + 1));
    int64_t *rank_b = (int64_t *)malloc(sizeof(int64_t) * (E + 1));
    int64_t *lp = (int64_t *)malloc(sizeof(int64_t) * (E + 2));
    int32_t *le = (int32_t *)malloc(sizeof(int32_t) * (E + 1));
    int64_t *lp_b = (int64_t *)malloc(sizeof(int64_t) * (E + 2));
    int32_t *le_b = (int32_t *)malloc(sizeof(int32_t) * (E + 1));
    int64_t *act = (int64_t *)malloc(sizeof(int64_t) * (E + 1));
    double *vres = (double *)malloc(sizeof(double) * (g->nv + 1));
    double *oldm = NULL;
    int64_t *ord = NULL;
    int64_t k = 0, k_b = 0, guards = 0, updates = 0;
    int rc = 0;
    if (!init) for (int64_t e = 0; e < 2 * E; e++) a2v[e] = 0.5;

    if (strategy == S_RESIDUAL) {
        ws.dres = (double *)calloc(E + 1, sizeof(double));
    } else {
        rc = orc_ranks(g, strategy == S_TOPO_FB ? S_TOPO : strategy, custom, 0, rank);
        if (rc == 0 && strategy == S_TOPO_FB) rc = orc_ranks(g, S_TOPO, custom, 1, rank_b);
        if (rc != 0) goto done;
        if (def2) {
            oldm = (double *)malloc(sizeof(double) * 2 * (E + 1));
            int64_t *all = (int64_t *)malloc(sizeof(int64_t) * (E + 1));
            for (int64_t e = 0; e < E; e++) all[e] = e;
            ord = canonical_order(rank, all, E);
            free(all);
        } else if (strategy == S_PARALL) {
            lp[0] = 0; lp[1] = E; k = E > 0;       /* one class: one level */
            for (int64_t e = 0; e < E; e++) le[e] = (int32_t)e;
        } else {
            k = orc_levels_nbr(g, rank, NULL, 0, lp, le);
            if (strategy == S_TOPO_FB) k_b = orc_levels_nbr(g, rank_b, NULL, 0, lp_b, le_b);
        }
    }

    int32_t it = 0;
    double res = 0.0;
    rc = 1;
    for (it = 1; it <= max_iters; it++) {
        res = 0.0;
        if (strategy == S_RESIDUAL) {
            int64_t n;
            if (it == 1) {
                for (int64_t e = 0; e < E; e++) { rank[e] = 0; act[e] = e; }
                n = E;
            } else {
                n = residual_active(g, ws.dres, tol, rank, act, vres);
            }
            for (int64_t e = 0; e < E; e++) ws.dres[e] = 0.0;
            k = orc_levels_nbr(g, rank, act, n, lp, le);
            run_levels(g, a2v, k, lp, le, &ws, &res, &guards);
            updates += n;
        } else if (def2) {
            run_def2(g, a2v, rank, ord, oldm, &ws, &res, &guards);
            updates += E;
        } else {
            run_levels(g, a2v, k, lp, le, &ws, &res, &guards);
            updates += E;
            if (strategy == S_TOPO_FB) {
                run_levels(g, a2v, k_b, lp_b, le_b, &ws, &res, &guards);
                updates += E;
            }
        }
        if (res_hist) res_hist[it - 1] = res;
        if (res < tol) { rc = 0; break; }
    }
    if (it > max_iters) it = max_iters;
    if (iters_out) *iters_out = it;
    if (residual_out) *residual_out = res;
done:
    if (min_pos_out) *min_pos_out = ws.min_pos;
    if (guards_out) *guards_out = guards;
    if (updates_out) *updates_out = updates;
    free(ws.v2a); free(ws.newm); free(ws.scratch); free(ws.mu); free(ws.fstamp); free(ws.vstamp);
    free(ws.dres); free(rank); free(rank_b); free(lp); free(le); free(lp_b); free(le_b);
    free(act); free(vres); free(oldm); free(ord);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Eq. (3): marginals P(x_v = 1) from the a->v messages and phi_v, with the  */
/* same zero-mass guard.  Returns the number of guarded variables.           */
/* ------------------------------------------------------------------------ */
int64_t orc_marginals(const og_graph *g, const double *a2v, double *p1)
{
    int64_t guards = 0;
    for (int32_t v = 0; v < g->nv; v++) {
        double m[2] = { g->phi[2 * v], g->phi[2 * v + 1] };
        for (int64_t k = g->vptr[v]; k < g->vptr[v + 1]; k++) {
            int64_t e = g->vedge[k];
            m[0] *= a2v[2 * e]; m[1] *= a2v[2 * e + 1];
            rescale(m);
        }
        guards += normalize_guard(m);
        p1[v] = m[1];
    }
    return guards;
}

/* One synchronous (PARALL) update of the listed edges from a given message
 * state: phase 1 then phase 2 for just those edges.  Lets the tests check a
 * sample of a full-size GPU iteration one message at a time. */
int orc_update_edges(const og_graph *g, const double *a2v, int64_t n, const int64_t *edges,
                     double *out)
{
    int bmax = 1;
    for (int64_t i = 0; i < n; i++) {
        int32_t a = g->efac[edges[i]];
        if (g->fptr[a + 1] - g->fptr[a] > bmax) bmax = (int)(g->fptr[a + 1] - g->fptr[a]);
    }
    double *v2a = (double *)malloc(sizeof(double) * 2 * (g->ne + 1));
    double *mu = (double *)malloc(sizeof(double) * 2 * (bmax + 1));
    for (int64_t i = 0; i < n; i++) {
        int64_t e = edges[i];
        int32_t a = g->efac[e];
        for (int64_t q = g->fptr[a]; q < g->fptr[a + 1]; q++)
            v2a_literal(g, a2v, g->fvars[q], q, v2a + 2 * q);
        a2v_alg1(g, v2a, e, out + 2 * i, mu);
    }
    free(v2a); free(mu);
    return 0;
}
