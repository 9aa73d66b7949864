/*
 * qai_oracle.c -- plain, slow FP64 CPU oracle of quantization-aware
 * interpolation (Jiao et al., "Mitigating Artifacts in Pre-quantization Based
 * Scientific Data Compressors with Quantization-aware Interpolation").
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. The CUDA
 * product path shares no code, header, table or helper with it.
 *
 * What it computes, step by step in the paper's order (Algorithm 4):
 *   A  GetBoundaryAndSignMap (Algorithm 2)          -> B1, S_B
 *   B  exact EDT of B1 with nearest-site index      -> Dist1, I1
 *      (Algorithm 1 applied along x, then y, then z)
 *   C  PropagateSignsAndConstructSignMap (Alg. 3)   -> S, B2
 *   D  exact EDT of B2 (distances only)             -> Dist2
 *   E  IDW compensation (Sec. VI step E)            -> C, D'' = D' + C
 * Integers stay integers (int64); every floating-point step is FP64.
 *
 * Readings where the paper is silent or ambiguous (each one is a named rule):
 *   R1  extent-1 axes are squeezed; the stencil uses the 2*rank axis
 *       neighbours of the remaining axes and "interior" means 1..d-2 on each.
 *   R2  sign_rule SUM (default): S_B = sgn(sum over neighbours of q_nb - q).
 *       sign_rule FIRST: sgn(q_nb - q) of the first differing neighbour in the
 *       order z-, z+, y-, y+, x-, x+.
 *   R3  the central difference of Algorithm 2 is (q[+1]-q[-1])/2 and its
 *       magnitude is compared, i.e. integer |q[+1]-q[-1]| >= grad_threshold
 *       (default 2 <=> |g| >= 1.0).
 *   R4  b2_rule SAME_Q (default): B2[i] iff some neighbour has the same q and
 *       a different S. b2_rule LITERAL: iff some neighbour has a different S.
 *   R5  ties in the nearest site: Algorithm 1's strict comparisons with the
 *       passes run x, then y, then z give the site with the smallest linear
 *       index among the nearest ones.
 *   R6  no site at all: distance INF (INT32_MAX on output), index -1, S = 0.
 *   R7  w = k2^p / (k1^p + k2^p); k1 = 0 -> w = 1 (takes precedence),
 *       k2 = 0 -> w = 0, k2 = INF -> w = 1. p = 1 is the paper's IDW.
 *   R8  k is the Euclidean distance, the square root of the EDT output.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_INF INT64_MAX

typedef struct {
    double eta;              /* compensation factor (paper: 0.9)            */
    double idw_power;        /* IDW exponent p (paper: 1)                   */
    int32_t grad_threshold;  /* R3, integer |q[+1]-q[-1]| threshold         */
    int32_t sign_rule;       /* R2: 0 = SUM, 1 = FIRST differing neighbour  */
    int32_t b2_rule;         /* R4: 0 = SAME_Q, 1 = LITERAL                 */
    uint32_t flags;          /* unused by the oracle                        */
} qai_oracle_params;

/* Canonical 3-D view after squeezing extent-1 axes (R1). n[2] is x, the
 * contiguous axis; axes with index < 3 - rank have extent 1. */
typedef struct {
    int rank;
    int64_t n[3];
    int64_t st[3];
    int64_t N;
} shape3;

static int make_shape(int rank, const int64_t* dims, shape3* s)
{
    int64_t kept[3];
    int r = 0;
    if (rank < 1 || rank > 3) return -1;
    for (int a = 0; a < rank; a++) {
        if (dims[a] < 1) return -1;
        if (dims[a] > 1) kept[r++] = dims[a];
    }
    if (r == 0) { kept[0] = 1; r = 1; }          /* a single point */
    s->rank = r;
    s->n[0] = s->n[1] = s->n[2] = 1;
    for (int a = 0; a < r; a++) s->n[3 - r + a] = kept[a];
    s->st[2] = 1;
    s->st[1] = s->n[2];
    s->st[0] = s->n[1] * s->n[2];
    s->N = s->n[0] * s->n[1] * s->n[2];
    return 0;
}

int qai_oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops from now on (n >= 1; timing only: the
 * results do not depend on it). */
void qai_oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int interior(const shape3* s, int64_t i)
{
    int64_t c[3] = { i / s->st[0], (i / s->st[1]) % s->n[1], i % s->n[2] };
    for (int a = 3 - s->rank; a < 3; a++)
        if (c[a] < 1 || c[a] > s->n[a] - 2) return 0;
    return 1;
}

static int sgn64(int64_t v) { return (v > 0) - (v < 0); }

/* ---- Step A: Algorithm 2, GetBoundaryAndSignMap ------------------------- */
void qai_oracle_boundary_and_sign(const int32_t* Q, int rank, const int64_t* dims,
                                  const qai_oracle_params* p, uint8_t* B, int8_t* S)
{
    shape3 s;
    if (make_shape(rank, dims, &s)) return;
    memset(B, 0, (size_t)s.N);
    memset(S, 0, (size_t)s.N);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s.N; i++) {
        if (!interior(&s, i)) continue;                 /* domain-edge points */
        int64_t q = Q[i];
        int differs = 0, first = 0;
        int64_t sum = 0;
        int zero_sign = 0;
        for (int a = 3 - s.rank; a < 3; a++) {          /* z, y, x order      */
            int64_t lo = Q[i - s.st[a]], hi = Q[i + s.st[a]];
            if (lo != q) { differs = 1; if (!first) first = sgn64(lo - q); }
            if (hi != q) { differs = 1; if (!first) first = sgn64(hi - q); }
            sum += (lo - q) + (hi - q);
            /* central difference g_a = (hi - lo) / 2; fast-varying if |g_a| >= 1 (R3) */
            int64_t d = hi - lo;
            if (d < 0) d = -d;
            if (d >= p->grad_threshold) zero_sign = 1;
        }
        if (!differs) continue;                         /* non-boundary       */
        B[i] = 1;
        int sign = (p->sign_rule == 1) ? first : sgn64(sum);
        S[i] = (int8_t)(zero_sign ? 0 : sign);
    }
}

/* ---- Steps B / D: Algorithm 1, VoronoiEDT along one line ---------------- */

/* RemoveEDT: parabola (g2,h2) is hidden by (g1,h1) and the new (f,i), i.e.
 * c*g2 - b*g1 - a*f - a*b*c > 0 with a = h2-h1, b = i-h2, c = i-h1. */
static int remove_edt(int64_t g1, int64_t g2, int64_t f, int64_t h1, int64_t h2, int64_t i)
{
    int64_t a = h2 - h1, b = i - h2, c = i - h1;
    return c * g2 - b * g1 - a * f - a * b * c > 0;
}

/* f[0..n): squared distances so far (ORC_INF = unreached); site[]: the site
 * index carried with each value. On return f[i] = min_j f[j] + (i-j)^2 over
 * the kept parabolas, the earliest one on ties, and site[i] its site. */
static void voronoi_edt_line(int64_t n, int64_t* f, int64_t* site,
                             int64_t* g, int64_t* h, int64_t* gs)
{
    int64_t l = 0;                                  /* parabolas on the stack */
    for (int64_t i = 0; i < n; i++) {               /* build partial Voronoi  */
        if (f[i] == ORC_INF) continue;
        while (l >= 2 && remove_edt(g[l - 2], g[l - 1], f[i], h[l - 2], h[l - 1], i)) l--;
        g[l] = f[i]; h[l] = i; gs[l] = site[i]; l++;
    }
    if (l == 0) return;                             /* no site on this line   */
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++) {               /* query the diagram      */
        while (k + 1 < l &&
               g[k] + (h[k] - i) * (h[k] - i) > g[k + 1] + (h[k + 1] - i) * (h[k + 1] - i))
            k++;
        f[i] = g[k] + (h[k] - i) * (h[k] - i);
        site[i] = gs[k];
    }
}

/* Exact squared EDT of a binary site map with the nearest site's linear index:
 * Algorithm 1 along x, then y, then z (R5). dist/idx are N-long int64. */
static void edt(const uint8_t* sites, const shape3* s, int64_t* dist, int64_t* idx)
{
    for (int64_t i = 0; i < s->N; i++) {
        dist[i] = sites[i] ? 0 : ORC_INF;
        idx[i] = sites[i] ? i : -1;
    }
    for (int a = 2; a >= 0; a--) {                  /* x, y, z                 */
        int64_t n = s->n[a], st = s->st[a];
        if (n == 1) continue;
        int64_t nlines = s->N / n;
        int b1 = (a == 0) ? 1 : 0, b2 = (a == 2) ? 1 : 2;   /* the other axes */
#pragma omp parallel
        {
            int64_t* buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)n * 5);
            int64_t *f = buf, *site = buf + n, *g = buf + 2 * n, *h = buf + 3 * n, *gs = buf + 4 * n;
#pragma omp for schedule(static)
            for (int64_t line = 0; line < nlines; line++) {
                int64_t u = line / s->n[b2], v = line % s->n[b2];
                int64_t base = u * s->st[b1] + v * s->st[b2];
                for (int64_t t = 0; t < n; t++) { f[t] = dist[base + t * st]; site[t] = idx[base + t * st]; }
                voronoi_edt_line(n, f, site, g, h, gs);
                for (int64_t t = 0; t < n; t++) { dist[base + t * st] = f[t]; idx[base + t * st] = site[t]; }
            }
            free(buf);
        }
    }
}

/* EDT entry point for tests: int32 outputs, INF -> INT32_MAX, no site -> -1. */
int qai_oracle_edt(const uint8_t* sites, int rank, const int64_t* dims,
                   int32_t* dist_out, int32_t* idx_out)
{
    shape3 s;
    if (make_shape(rank, dims, &s)) return -1;
    int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)s.N);
    int64_t* x = (int64_t*)malloc(sizeof(int64_t) * (size_t)s.N);
    if (!d || !x) { free(d); free(x); return -2; }
    edt(sites, &s, d, x);
    for (int64_t i = 0; i < s.N; i++) {
        dist_out[i] = d[i] == ORC_INF ? INT32_MAX : (int32_t)d[i];
        if (idx_out) idx_out[i] = (int32_t)x[i];
    }
    free(d); free(x);
    return 0;
}

/* ---- Step C: Algorithm 3, PropagateSignsAndConstructSignMap ------------- */

/* GetBoundary(S) with the R4 rule, interior points only (as in Alg. 2). */
static void boundary_of_s(const int32_t* Q, const shape3* s, const qai_oracle_params* p,
                          const int8_t* S, uint8_t* B2)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s->N; i++) {
        B2[i] = 0;
        if (!interior(s, i)) continue;
        for (int a = 3 - s->rank; a < 3; a++) {
            int64_t nb[2] = { i - s->st[a], i + s->st[a] };
            for (int k = 0; k < 2; k++) {
                if (p->b2_rule == 0 && Q[nb[k]] != Q[i]) continue;
                if (S[nb[k]] != S[i]) B2[i] = 1;
            }
        }
    }
}

static void propagate_and_b2(const int32_t* Q, const shape3* s, const qai_oracle_params* p,
                             const uint8_t* B1, const int8_t* SB, const int64_t* I1,
                             int8_t* S, uint8_t* B2)
{
    memcpy(S, SB, (size_t)s->N);
    /* In place is safe: S is only read at boundary points, never written there. */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s->N; i++)
        if (B1[i] != 1) S[i] = (I1[i] >= 0) ? S[I1[i]] : 0;
    boundary_of_s(Q, s, p, S, B2);
}

/* GetBoundary(S) alone (the second half of Algorithm 3) for a given S. */
int qai_oracle_boundary_of_s(const int32_t* Q, const int8_t* S, int rank, const int64_t* dims,
                             const qai_oracle_params* p, uint8_t* B2)
{
    shape3 s;
    if (make_shape(rank, dims, &s)) return -1;
    boundary_of_s(Q, &s, p, S, B2);
    return 0;
}

/* ---- Step E: IDW compensation ------------------------------------------- */
static double idw_weight(int64_t d1, int64_t d2, double pw)
{
    if (d1 == 0) return 1.0;                /* on a quantization boundary     */
    if (d2 == 0) return 0.0;                /* on a sign-flipping boundary    */
    if (d2 == ORC_INF) return 1.0;          /* limit of the formula, k2 -> oo */
    if (d1 == ORC_INF) return 0.0;          /* no boundary at all: S = 0      */
    double k1 = sqrt((double)d1), k2 = sqrt((double)d2);
    /* (1/k1^p) / (1/k1^p + 1/k2^p) written as k2^p / (k1^p + k2^p) */
    double a = pow(k1, pw), b = pow(k2, pw);
    return b / (a + b);
}

/* Step E at n points: D' = 2 q eps (Eq. 1), C = S w eta eps, out = D' + C. */
static void compensate(const int32_t* Q, const int64_t* D1, const int64_t* D2, const int8_t* S,
                       int64_t n, double eb, const qai_oracle_params* p, double* out, double* comp_out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double dprime = 2.0 * (double)Q[i] * eb;
        double c = (double)S[i] * idw_weight(D1[i], D2[i], p->idw_power) * p->eta * eb;
        if (out) out[i] = dprime + c;
        if (comp_out) comp_out[i] = c;
    }
}

/* Step E alone on given int32 distances (INT32_MAX = INF) and S. */
int qai_oracle_compensate(const int32_t* Q, const int32_t* dist1, const int32_t* dist2, const int8_t* S,
                          int64_t n, double eb, const qai_oracle_params* p, double* out)
{
    if (n < 0 || !(eb > 0.0) || !isfinite(eb)) return -1;
    int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * n + 1));
    if (!d) return -2;
    for (int64_t i = 0; i < n; i++) {
        d[i] = dist1[i] == INT32_MAX ? ORC_INF : dist1[i];
        d[n + i] = dist2[i] == INT32_MAX ? ORC_INF : dist2[i];
    }
    compensate(Q, d, d + n, S, n, eb, p, out, NULL);
    free(d);
    return 0;
}

/* Full Algorithm 4. out = D'' (FP64). Every other pointer may be NULL. */
int qai_oracle_mitigate(const int32_t* Q, int rank, const int64_t* dims, double eb,
                        const qai_oracle_params* p, double* out,
                        uint8_t* b1_out, int8_t* sb_out, int32_t* dist1_out,
                        int32_t* idx1_out, int8_t* s_out, uint8_t* b2_out,
                        int32_t* dist2_out, double* comp_out)
{
    shape3 s;
    if (make_shape(rank, dims, &s)) return -1;
    if (!(eb > 0.0) || !isfinite(eb)) return -1;
    size_t N = (size_t)s.N;
    uint8_t* B1 = (uint8_t*)malloc(N);
    int8_t* SB = (int8_t*)malloc(N);
    int8_t* S = (int8_t*)malloc(N);
    uint8_t* B2 = (uint8_t*)malloc(N);
    int64_t* D1 = (int64_t*)malloc(N * 8);
    int64_t* I1 = (int64_t*)malloc(N * 8);
    int64_t* D2 = (int64_t*)malloc(N * 8);
    int64_t* I2 = (int64_t*)malloc(N * 8);
    int rc = 0;
    if (!B1 || !SB || !S || !B2 || !D1 || !I1 || !D2 || !I2) { rc = -2; goto done; }

    qai_oracle_boundary_and_sign(Q, rank, dims, p, B1, SB);      /* step A */
    edt(B1, &s, D1, I1);                                          /* step B */
    propagate_and_b2(Q, &s, p, B1, SB, I1, S, B2);                /* step C */
    edt(B2, &s, D2, I2);                                          /* step D */

    compensate(Q, D1, D2, S, s.N, eb, p, out, comp_out);          /* step E */
    for (int64_t i = 0; i < s.N; i++) {
        if (b1_out) b1_out[i] = B1[i];
        if (sb_out) sb_out[i] = SB[i];
        if (s_out) s_out[i] = S[i];
        if (b2_out) b2_out[i] = B2[i];
        if (dist1_out) dist1_out[i] = D1[i] == ORC_INF ? INT32_MAX : (int32_t)D1[i];
        if (idx1_out) idx1_out[i] = (int32_t)I1[i];
        if (dist2_out) dist2_out[i] = D2[i] == ORC_INF ? INT32_MAX : (int32_t)D2[i];
    }
done:
    free(B1); free(SB); free(S); free(B2); free(D1); free(I1); free(D2); free(I2);
    return rc;
}

/* ---- Section VII-B, approximate parallelization -------------------------
 * The field (rank 2 or 3 after R1) is cut along its slowest axis into nparts
 * slabs, slab k holding the planes [floor(k n0 / P), floor((k + 1) n0 / P)).
 * Each part exchanges one ghost plane with each neighbour before step A and
 * again (its S) before the boundary of step C; both EDTs stay inside the
 * part. So, per part, in the paper's order:
 *   A  B1, S_B: with q's ghost planes the stencil is the whole field's, so
 *      they are the whole-field maps restricted to the part;
 *   B  exact EDT of the part's own B1 points over the part's points only;
 *   C  S = S_B[I1] with that local I1; then, with S's ghost planes from the
 *      neighbours' own local S, B2 = GetBoundary(S) with the whole field's
 *      interior rule;
 *   D  exact EDT of the part's own B2 points over the part's points only;
 *   E  as in Algorithm 4.
 * idx1 is returned as a linear index of the whole field. nparts = 1 is
 * Algorithm 4 itself. */
static void slab_range(int k, int nparts, int64_t n0, int64_t* z0, int64_t* z1)
{
    *z0 = k * n0 / nparts;
    *z1 = (k + 1) * n0 / nparts;
}

static void slab_shape(const shape3* s, int64_t z0, int64_t z1, shape3* sl)
{
    *sl = *s;
    sl->n[3 - s->rank] = z1 - z0;
    sl->st[2] = 1;
    sl->st[1] = sl->n[2];
    sl->st[0] = sl->n[1] * sl->n[2];
    sl->N = sl->n[0] * sl->n[1] * sl->n[2];
}

int qai_oracle_mitigate_approx(const int32_t* Q, int rank, const int64_t* dims, double eb,
                               const qai_oracle_params* p, int nparts, double* out,
                               int32_t* dist1_out, int32_t* idx1_out, int8_t* s_out,
                               uint8_t* b2_out, int32_t* dist2_out)
{
    shape3 s;
    if (make_shape(rank, dims, &s)) return -1;
    if (s.rank < 2 || !(eb > 0.0) || !isfinite(eb)) return -1;
    const int ax = 3 - s.rank;                       /* the slab axis          */
    const int64_t n0 = s.n[ax], plane = s.st[ax];
    if (nparts < 1 || nparts > n0) return -1;
    size_t N = (size_t)s.N;
    uint8_t* B1 = (uint8_t*)malloc(N);
    int8_t* SB = (int8_t*)malloc(N);
    int8_t* S = (int8_t*)malloc(N);
    uint8_t* B2 = (uint8_t*)malloc(N);
    int64_t* D1 = (int64_t*)malloc(N * 8);
    int64_t* I1 = (int64_t*)malloc(N * 8);
    int64_t* D2 = (int64_t*)malloc(N * 8);
    int64_t* I2 = (int64_t*)malloc(N * 8);
    int rc = 0;
    if (!B1 || !SB || !S || !B2 || !D1 || !I1 || !D2 || !I2) { rc = -2; goto done; }

    qai_oracle_boundary_and_sign(Q, rank, dims, p, B1, SB);      /* step A */
    for (int k = 0; k < nparts; k++) {                            /* steps B, C (S) */
        int64_t z0, z1;
        slab_range(k, nparts, n0, &z0, &z1);
        const int64_t off = z0 * plane;
        shape3 sl;
        slab_shape(&s, z0, z1, &sl);
        edt(B1 + off, &sl, D1 + off, I1 + off);
        for (int64_t i = off; i < off + sl.N; i++) {
            if (I1[i] >= 0) I1[i] += off;                         /* whole-field index */
            S[i] = B1[i] ? SB[i] : (I1[i] >= 0 ? SB[I1[i]] : 0);
        }
    }
    boundary_of_s(Q, &s, p, S, B2);                               /* step C (B2) */
    for (int k = 0; k < nparts; k++) {                            /* step D */
        int64_t z0, z1;
        slab_range(k, nparts, n0, &z0, &z1);
        const int64_t off = z0 * plane;
        shape3 sl;
        slab_shape(&s, z0, z1, &sl);
        edt(B2 + off, &sl, D2 + off, I2 + off);
    }
    compensate(Q, D1, D2, S, s.N, eb, p, out, NULL);              /* step E */
    for (int64_t i = 0; i < s.N; i++) {
        if (s_out) s_out[i] = S[i];
        if (b2_out) b2_out[i] = B2[i];
        if (dist1_out) dist1_out[i] = D1[i] == ORC_INF ? INT32_MAX : (int32_t)D1[i];
        if (idx1_out) idx1_out[i] = (int32_t)I1[i];
        if (dist2_out) dist2_out[i] = D2[i] == ORC_INF ? INT32_MAX : (int32_t)D2[i];
    }
done:
    free(B1); free(SB); free(S); free(B2); free(D1); free(I1); free(D2); free(I2);
    return rc;
}

/* ---- Adjoint of step E (no counterpart in the paper) ---------------------
 * With the EDT assignment held fixed (Dist1, Dist2, S from Algorithm 4),
 * D'' = D' + S w(k1, k2; p) eta eps. For a loss L with dL/dD'' = G:
 *   dL/deta = sum_i G_i S_i w_i eps
 *   dL/dp   = sum_i G_i S_i eta eps dw_i/dp,
 *   dw/dp   = w (1 - w) (ln k2 - ln k1) for finite k1, k2 > 0, else 0
 * (w = 1 / (1 + (k1/k2)^p)). dL/dD' = G. FP64 throughout. */
int qai_oracle_grad_params(const int32_t* Q, int rank, const int64_t* dims, double eb,
                           const qai_oracle_params* p, const double* G, double* grad /*[2]*/)
{
    shape3 s;
    if (make_shape(rank, dims, &s)) return -1;
    size_t N = (size_t)s.N;
    int32_t* d1 = (int32_t*)malloc(N * 4);
    int32_t* d2 = (int32_t*)malloc(N * 4);
    int8_t* S = (int8_t*)malloc(N);
    int rc = 0;
    if (!d1 || !d2 || !S) { rc = -2; goto done; }
    rc = qai_oracle_mitigate(Q, rank, dims, eb, p, NULL, NULL, NULL, d1, NULL, S, NULL, d2, NULL);
    if (rc) goto done;
    double ge = 0.0, gp = 0.0;
    for (int64_t i = 0; i < s.N; i++) {
        if (S[i] == 0) continue;
        int64_t a = d1[i] == INT32_MAX ? ORC_INF : d1[i];
        int64_t b = d2[i] == INT32_MAX ? ORC_INF : d2[i];
        double w = idw_weight(a, b, p->idw_power);
        ge += G[i] * S[i] * w * eb;
        if (a > 0 && b > 0 && a != ORC_INF && b != ORC_INF) {
            double dw = w * (1.0 - w) * (0.5 * log((double)b) - 0.5 * log((double)a));
            gp += G[i] * S[i] * p->eta * eb * dw;
        }
    }
    grad[0] = ge;
    grad[1] = gp;
done:
    free(d1); free(d2); free(S);
    return rc;
}
