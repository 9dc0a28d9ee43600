/*
 * tvs_oracle.c -- the oracle: a plain, slow CPU restatement of the sDEM total
 * viewshed (Sanchez-Fernandez, Romero, Bandera, Tabik, arXiv 2003.02200).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  The product library never
 * links, loads or calls it, and it shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * What it computes (all in the paper's notation, section 3 and 4.1):
 *
 *  - Every DEM cell is a POV lifted by h0 (Alg. 1).  The half-plane of
 *    directions is cut into n "directions" theta_k = k*pi/n, k = 0..n-1; each
 *    direction is walked forward and backward (step 1(c)i of the methodology in
 *    section 4.1: sectors s and s+180 deg), so there are 2n half-line sectors of
 *    angular width pi/n and the Pappus factor of Alg. 1 becomes pi/(2n)
 *    (for n = 180 this is the pi/360 of the ring-sector area equation).
 *  - Lines of sight are sampled the way Kernel-1 (Alg. 6) samples them: along
 *    the major axis j, the minor coordinate is y = b + j*tan(alpha), split into
 *    an integer part dest and a fraction r, and the height is the linear blend
 *    (1-r)*V[a][j] + r*V[a+1][j].  tan(alpha) is held in 32.32 fixed point so
 *    that every offset is an exact integer.
 *  - Alg. 6 only covers 0 <= s <= 45 deg.  The other three eighths of the
 *    half-plane reuse it through a D4 view of the DEM (identity, transpose,
 *    transpose+column mirror, row mirror), picked by integer tests on k.
 *  - A DEM cell lies between two sampled lines: the one through fractional row
 *    i + r(j0) (weight 1-r) and the one through i - 1 + r(j0) (weight r), the
 *    interpolation weights of Kernel-3 (Alg. 9).  A line whose sample at j0
 *    falls outside the DEM is dropped and the other one takes weight 1.
 *  - A walk follows Alg. 8 with the readings stated in-line below: slope
 *    theta = (z - h)/dd, a target is visible iff theta > max theta (strict),
 *    a visible segment opens at the first visible target and closes at the
 *    first hidden one, adding dd^2 - open^2; a segment still open at the end of
 *    the line closes at the last target.  The walk visits every valid sample of
 *    the line up to dd <= K (a max-range cap, unlimited by default).
 *  - The cell's value is g * sum(w * cv) summed over directions, with
 *    g = 1 + t^2 the (1/cos s)^2 distance factor of Alg. 7 (t the fixed-point
 *    tangent), scaled once by (pi/(2n)) * step^2 (Pappus, ring-sector area).
 *
 * There is no skewed array here: every walk is taken directly in DEM (view)
 * coordinates, one cell and one direction at a time.
 *
 * Besides the total viewshed (orc_total_viewshed and its per-direction and
 * per-line detail), the oracle holds the singular viewshed by definition
 * (orc_direct_viewshed: lines of sight through the POV cell itself, Alg. 1-3)
 * and the visibility map of a list of POVs (orc_visibility_map).
 *
 * Precision.  prec = 64 computes heights and slopes in double precision with a
 * true division.  prec = 32 takes every height and slope in single precision,
 * as the paper's kernels declare them ("float" in Alg. 6, 7 and 8): the blend
 * is (1-r)*a + r*b with r = float(frac) * 2^-32, h = z + float(h0), and
 * theta = (z - h) * rcp(dd) with rcp(dd) = 1.0f/dd correctly rounded.  Only
 * the visibility decisions change with prec; cv stays an exact integer and all
 * sums are double in both modes.
 *
 * Build: plain C99, -O2 -fopenmp -ffp-contract=off (no fused multiply-add, so
 * the result is the same on x86-64 and AArch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-2)

#define TWO32 4294967296.0

/* One direction k of n: its D4 view, fixed-point tangent and walk limit. */
typedef struct {
    int frame;        /* 0 identity, 1 transpose, 2 transpose+mirror cols, 3 mirror rows */
    int m;            /* reduced angle alpha = pi*m/(2n), 0 <= alpha <= pi/4 */
    int H, W;         /* shape of the view: W is the walk (major) axis */
    uint64_t t_fx;    /* llround(tan(alpha) * 2^32), 0 .. 2^32 */
    double t;         /* t_fx * 2^-32 */
    double g;         /* 1 + t^2: squared length of one major-axis step */
    int64_t K;        /* max steps per walk (INT64_MAX = unlimited) */
    int64_t D;        /* dest(W-1): how far the last column is shifted */
} orc_dir;

/* Direction k of n (section 4.1 step 1, Alg. 6 for 0..45 deg, extended by D4
 * symmetry).  theta_k = k*pi/n measured from +j (east) toward +i (south). */
int orc_direction(int n, int k, int rows, int cols, double step, double max_range,
                  orc_dir* d)
{
    if (!d || n < 1 || k < 0 || k >= n || rows < 2 || cols < 2) return ORC_ERR_ARG;
    if (!(step > 0.0) || isnan(max_range)) return ORC_ERR_ARG;
    memset(d, 0, sizeof(*d));
    int64_t k4 = 4 * (int64_t)k;
    if (k4 < n)          { d->frame = 0; d->m = 2 * k;         d->H = rows; d->W = cols; }
    else if (k4 < 2 * (int64_t)n) { d->frame = 1; d->m = n - 2 * k;     d->H = cols; d->W = rows; }
    else if (k4 < 3 * (int64_t)n) { d->frame = 2; d->m = 2 * k - n;     d->H = cols; d->W = rows; }
    else                 { d->frame = 3; d->m = 2 * n - 2 * k; d->H = rows; d->W = cols; }
    double alpha = M_PI * (double)d->m / (2.0 * (double)n);
    d->t_fx = (uint64_t)llround(tan(alpha) * TWO32);
    d->t = (double)d->t_fx / TWO32;
    d->g = 1.0 + d->t * d->t;
    if (!(max_range > 0.0) || isinf(max_range)) {
        d->K = INT64_MAX;
    } else {
        double kk = floor(max_range / (step * sqrt(d->g)));
        d->K = kk >= 9.0e18 ? INT64_MAX : (int64_t)kk;
    }
    d->D = (int64_t)(((uint64_t)(d->W - 1) * d->t_fx) >> 32);
    return ORC_OK;
}

/* Value of the view V (H x W) at (i, j), read from the row-major DEM. */
static inline float view_at(const float* dem, int cols, const orc_dir* d, int64_t i, int64_t j)
{
    switch (d->frame) {
    case 0:  return dem[i * cols + j];
    case 1:  return dem[j * cols + i];
    case 2:  return dem[(d->W - 1 - j) * cols + i];
    default: return dem[(d->H - 1 - i) * cols + j];
    }
}

/* Position of the sample of line b at column j: integer row a, fraction fr/2^32. */
static inline void sample_pos(const orc_dir* d, int64_t b, int64_t j, int64_t* a, uint32_t* fr)
{
    uint64_t y = (uint64_t)j * d->t_fx;
    *a = b + (int64_t)(y >> 32);
    *fr = (uint32_t)(y & 0xFFFFFFFFu);
}

/* A sample is usable iff both rows it blends lie inside the DEM (a sample with
 * r = 0 needs only row a).  This replaces the paper's "non-zero" nzSet test,
 * which would drop real 0 m elevations and keep half-outside blends. */
static inline int sample_ok(const orc_dir* d, int64_t b, int64_t j)
{
    if (j < 0 || j >= d->W) return 0;
    int64_t a; uint32_t fr;
    sample_pos(d, b, j, &a, &fr);
    if (a < 0) return 0;
    return fr == 0 ? (a <= d->H - 1) : (a + 1 <= d->H - 1);
}

static inline double sample64(const float* dem, int cols, const orc_dir* d, int64_t b, int64_t j)
{
    int64_t a; uint32_t fr;
    sample_pos(d, b, j, &a, &fr);
    if (fr == 0) return (double)view_at(dem, cols, d, a, j);
    double r = (double)fr / TWO32;
    double lo = (double)view_at(dem, cols, d, a, j);
    double hi = (double)view_at(dem, cols, d, a + 1, j);
    return (1.0 - r) * lo + r * hi;
}

static inline float sample32(const float* dem, int cols, const orc_dir* d, int64_t b, int64_t j)
{
    int64_t a; uint32_t fr;
    sample_pos(d, b, j, &a, &fr);
    if (fr == 0) return view_at(dem, cols, d, a, j);
    float r = (float)fr * 0x1p-32f;
    float wa = 1.0f - r;
    float pa = wa * view_at(dem, cols, d, a, j);
    float pb = r * view_at(dem, cols, d, a + 1, j);
    return pa + pb;
}

/*
 * One linear viewshed (Alg. 2 / Alg. 8) along line b from column j0 in
 * direction dir (+1 forward, -1 backward), observer height h.  Readings:
 *   - visible starts true and max theta at -inf (Alg. 2), so the POV's own
 *     ring [0,1) is visible and the first target keeps the segment open;
 *   - "above" is recomputed for every target (Alg. 8 never resets it);
 *   - theta = (target - observer)/dd (Alg. 8's sign; Alg. 3's is reversed);
 *   - a segment still open when the line ends closes at the last target.
 * Returns cv, the visible measure in squared steps (an exact integer).
 */
static int64_t walk64(const float* dem, int cols, const orc_dir* d, int64_t b, int64_t j0,
                      int dir, double h, int64_t* nev)
{
    int vis = 1;
    int64_t open = 0, last = 0, cv = 0;
    double maxth = -INFINITY;
    for (int64_t dd = 1; dd <= d->K; ++dd) {
        int64_t j = j0 + dir * dd;
        if (!sample_ok(d, b, j)) break;
        double th = (sample64(dem, cols, d, b, j) - h) / (double)dd;
        int above = th > maxth;
        if (above && !vis) open = dd;
        if (!above && vis) cv += dd * dd - open * open;
        vis = above;
        if (th > maxth) maxth = th;
        last = dd;
    }
    if (vis) cv += last * last - open * open;
    if (nev) *nev += last;
    return cv;
}

static int64_t walk32(const float* dem, int cols, const orc_dir* d, int64_t b, int64_t j0,
                      int dir, float h, const float* rcp, int64_t* nev)
{
    int vis = 1;
    int64_t open = 0, last = 0, cv = 0;
    float maxth = -INFINITY;
    for (int64_t dd = 1; dd <= d->K; ++dd) {
        int64_t j = j0 + dir * dd;
        if (!sample_ok(d, b, j)) break;
        float diff = sample32(dem, cols, d, b, j) - h;
        float th = diff * rcp[dd];
        int above = th > maxth;
        if (above && !vis) open = dd;
        if (!above && vis) cv += dd * dd - open * open;
        vis = above;
        if (th > maxth) maxth = th;
        last = dd;
    }
    if (vis) cv += last * last - open * open;
    if (nev) *nev += last;
    return cv;
}

/* View coordinates (i, j) of DEM cell (iD, jD) under direction d. */
static inline void to_view(const orc_dir* d, int64_t iD, int64_t jD, int64_t* i, int64_t* j)
{
    switch (d->frame) {
    case 0:  *i = iD;             *j = jD;             break;
    case 1:  *i = jD;             *j = iD;             break;
    case 2:  *i = jD;             *j = d->W - 1 - iD;  break;
    default: *i = d->H - 1 - iD;  *j = jD;             break;
    }
}

/* The virtual POVs of view cell (i, j): base lines b[] and weights w[] (Alg. 9). */
static int virtual_povs(const orc_dir* d, int64_t i, int64_t j, int64_t b[2], double w[2])
{
    uint64_t y = (uint64_t)j * d->t_fx;
    int64_t dest = (int64_t)(y >> 32);
    uint32_t fr = (uint32_t)(y & 0xFFFFFFFFu);
    if (fr == 0) { b[0] = i - dest; w[0] = 1.0; return 1; }
    double r = (double)fr / TWO32;
    int hi_ok = i <= d->H - 2;     /* line through i + r: needs rows i, i+1 */
    int lo_ok = i >= 1;            /* line through i - 1 + r: needs rows i-1, i */
    if (hi_ok && lo_ok) {
        b[0] = i - dest;     w[0] = 1.0 - r;
        b[1] = i - dest - 1; w[1] = r;
        return 2;
    }
    if (hi_ok) { b[0] = i - dest;     w[0] = 1.0; return 1; }
    b[0] = i - dest - 1; w[0] = 1.0; return 1;
}

typedef struct {
    const float* dem; int rows, cols; double step, h0; int n; int prec;
    orc_dir* dirs; float* rcp; int64_t maxd;
} orc_ctx;

static int ctx_init(orc_ctx* c, const float* dem, int rows, int cols, double step, double h0,
                    int n, double max_range, int prec)
{
    if (!dem || rows < 2 || cols < 2 || n < 1 || !(step > 0.0) || !isfinite(step)) return ORC_ERR_ARG;
    if (!isfinite(h0) || isnan(max_range) || (prec != 32 && prec != 64)) return ORC_ERR_ARG;
    for (int64_t q = 0; q < (int64_t)rows * cols; ++q)
        if (!isfinite(dem[q])) return ORC_ERR_ARG;
    memset(c, 0, sizeof(*c));
    c->dem = dem; c->rows = rows; c->cols = cols; c->step = step; c->h0 = h0; c->n = n; c->prec = prec;
    c->dirs = (orc_dir*)malloc(sizeof(orc_dir) * (size_t)n);
    c->maxd = (rows > cols ? rows : cols) + 1;
    c->rcp = (float*)malloc(sizeof(float) * (size_t)(c->maxd + 1));
    if (!c->dirs || !c->rcp) { free(c->dirs); free(c->rcp); return ORC_ERR_OOM; }
    for (int k = 0; k < n; ++k) orc_direction(n, k, rows, cols, step, max_range, &c->dirs[k]);
    c->rcp[0] = 0.0f;
    for (int64_t q = 1; q <= c->maxd; ++q) c->rcp[q] = 1.0f / (float)q;
    return ORC_OK;
}

static void ctx_free(orc_ctx* c) { free(c->dirs); free(c->rcp); }

/* Sum over directions of g * sum_v w_v * (cv_fwd + cv_bwd) for one DEM cell. */
static double cell_acc(const orc_ctx* c, int64_t iD, int64_t jD, int64_t* nev)
{
    double acc = 0.0;
    for (int k = 0; k < c->n; ++k) {
        const orc_dir* d = &c->dirs[k];
        int64_t i, j, b[2]; double w[2];
        to_view(d, iD, jD, &i, &j);
        int nv = virtual_povs(d, i, j, b, w);
        double part = 0.0;
        for (int v = 0; v < nv; ++v) {
            int64_t cv;
            if (c->prec == 64) {
                double h = sample64(c->dem, c->cols, d, b[v], j) + c->h0;
                cv = walk64(c->dem, c->cols, d, b[v], j, +1, h, nev)
                   + walk64(c->dem, c->cols, d, b[v], j, -1, h, nev);
            } else {
                float h = sample32(c->dem, c->cols, d, b[v], j) + (float)c->h0;
                cv = walk32(c->dem, c->cols, d, b[v], j, +1, h, c->rcp, nev)
                   + walk32(c->dem, c->cols, d, b[v], j, -1, h, c->rcp, nev);
            }
            part += w[v] * (double)cv;
        }
        acc += d->g * part;
    }
    return acc;
}

static double pappus_scale(int n, double step) { return (M_PI / (2.0 * (double)n)) * (step * step); }

/*
 * Total viewshed (Alg. 4) of the cells listed in idx (row-major linear indices;
 * idx == NULL means all rows*cols cells, in order).  out[q] is the visible
 * area of cell idx[q] in the squared unit of step (m^2 for step in metres).
 * nthreads <= 0 uses the OpenMP default.  *threads_used (optional) reports the
 * team size, *evals_visited (optional) the number of targets the walks visited.
 */
int orc_total_viewshed(const float* dem, int rows, int cols, double step, double h0, int n,
                       double max_range, int prec, const int64_t* idx, int64_t count,
                       double* out, int nthreads, int* threads_used, int64_t* evals_visited)
{
    orc_ctx c;
    int rc = ctx_init(&c, dem, rows, cols, step, h0, n, max_range, prec);
    if (rc) return rc;
    if (!out) { ctx_free(&c); return ORC_ERR_ARG; }
    int64_t total = idx ? count : (int64_t)rows * cols;
    if (idx)
        for (int64_t q = 0; q < count; ++q)
            if (idx[q] < 0 || idx[q] >= (int64_t)rows * cols) { ctx_free(&c); return ORC_ERR_ARG; }
    double scale = pappus_scale(n, step);
    int64_t nev = 0;
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(+ : nev)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 8)
        for (int64_t q = 0; q < total; ++q) {
            int64_t cell = idx ? idx[q] : q;
            out[q] = scale * cell_acc(&c, cell / cols, cell % cols, &nev);
        }
    }
#else
    (void)nthreads;
    for (int64_t q = 0; q < total; ++q) {
        int64_t cell = idx ? idx[q] : q;
        out[q] = scale * cell_acc(&c, cell / cols, cell % cols, &nev);
    }
#endif
    if (threads_used) *threads_used = used;
    if (evals_visited) *evals_visited = nev;
    ctx_free(&c);
    return ORC_OK;
}

/*
 * Per-direction detail of one DEM cell: for direction k, the number of virtual
 * POVs (1 or 2), their base lines b, weights w and cv (forward, backward).
 */
int orc_cell_direction(const float* dem, int rows, int cols, double step, double h0, int n,
                       double max_range, int prec, int iD, int jD, int k,
                       int* npov, int64_t* b_out, double* w_out, int64_t* cv_fwd, int64_t* cv_bwd)
{
    if (iD < 0 || iD >= rows || jD < 0 || jD >= cols || k < 0 || k >= n) return ORC_ERR_ARG;
    orc_ctx c;
    int rc = ctx_init(&c, dem, rows, cols, step, h0, n, max_range, prec);
    if (rc) return rc;
    const orc_dir* d = &c.dirs[k];
    int64_t i, j, b[2]; double w[2];
    to_view(d, iD, jD, &i, &j);
    int nv = virtual_povs(d, i, j, b, w);
    *npov = nv;
    for (int v = 0; v < nv; ++v) {
        b_out[v] = b[v]; w_out[v] = w[v];
        if (prec == 64) {
            double h = sample64(dem, cols, d, b[v], j) + h0;
            cv_fwd[v] = walk64(dem, cols, d, b[v], j, +1, h, NULL);
            cv_bwd[v] = walk64(dem, cols, d, b[v], j, -1, h, NULL);
        } else {
            float h = sample32(dem, cols, d, b[v], j) + (float)h0;
            cv_fwd[v] = walk32(dem, cols, d, b[v], j, +1, h, c.rcp, NULL);
            cv_bwd[v] = walk32(dem, cols, d, b[v], j, -1, h, c.rcp, NULL);
        }
    }
    ctx_free(&c);
    return ORC_OK;
}

/*
 * cv (forward + backward) of the POV at column j of line b, direction k, for
 * every usable sample of that line: out[j] for j in [0, W), -1 where the sample
 * is not usable.  This is the per-line quantity the skewed layout stores.
 */
int orc_line_cv(const float* dem, int rows, int cols, double step, double h0, int n,
                double max_range, int prec, int k, int64_t b, int64_t* out, int W_cap)
{
    if (k < 0 || k >= n || !out) return ORC_ERR_ARG;
    orc_ctx c;
    int rc = ctx_init(&c, dem, rows, cols, step, h0, n, max_range, prec);
    if (rc) return rc;
    const orc_dir* d = &c.dirs[k];
    if (W_cap < d->W) { ctx_free(&c); return ORC_ERR_ARG; }
    for (int64_t j = 0; j < d->W; ++j) {
        if (!sample_ok(d, b, j)) { out[j] = -1; continue; }
        if (prec == 64) {
            double h = sample64(dem, cols, d, b, j) + h0;
            out[j] = walk64(dem, cols, d, b, j, +1, h, NULL) + walk64(dem, cols, d, b, j, -1, h, NULL);
        } else {
            float h = sample32(dem, cols, d, b, j) + (float)h0;
            out[j] = walk32(dem, cols, d, b, j, +1, h, c.rcp, NULL)
                   + walk32(dem, cols, d, b, j, -1, h, c.rcp, NULL);
        }
    }
    ctx_free(&c);
    return ORC_OK;
}

/* Usable column range [jlo, jhi] of line b (jlo > jhi when empty), found by
 * scanning the sample predicate (the set is contiguous because the sampled row
 * b + j*t never decreases in j). */
int orc_line_range(int n, int k, int rows, int cols, int64_t b, int64_t* jlo, int64_t* jhi)
{
    orc_dir d;
    int rc = orc_direction(n, k, rows, cols, 1.0, 0.0, &d);
    if (rc) return rc;
    int64_t lo = -1, hi = -2;
    for (int64_t j = 0; j < d.W; ++j) {
        if (sample_ok(&d, b, j)) { if (lo < 0) lo = j; hi = j; }
        else if (lo >= 0) break;
    }
    if (lo < 0) { lo = 0; hi = -1; }
    /* contiguity check: nothing usable after the run */
    for (int64_t j = hi + 1; j < d.W && hi >= 0; ++j)
        if (sample_ok(&d, b, j)) return ORC_ERR_ARG;
    *jlo = lo; *jhi = hi;
    return ORC_OK;
}

/* dest(j) and frac(j) (the 32-bit fraction) of direction k for every column. */
int orc_column_offsets(int n, int k, int rows, int cols, int64_t* dest, uint32_t* frac, int W_cap)
{
    orc_dir d;
    int rc = orc_direction(n, k, rows, cols, 1.0, 0.0, &d);
    if (rc) return rc;
    if (W_cap < d.W) return ORC_ERR_ARG;
    for (int64_t j = 0; j < d.W; ++j) {
        uint64_t y = (uint64_t)j * d.t_fx;
        dest[j] = (int64_t)(y >> 32);
        frac[j] = (uint32_t)(y & 0xFFFFFFFFu);
    }
    return ORC_OK;
}

static int64_t sum_min(int64_t L, int64_t K)
{
    /* sum_{x=0}^{L-1} min(x, K) */
    if (L <= 0) return 0;
    if (L - 1 <= K) return (L - 1) * L / 2;
    return K * (K + 1) / 2 + (L - 1 - K) * K;
}

/*
 * Work count: the number of (virtual POV, direction, target) visits of the
 * skewed formulation, sum over directions, lines and usable samples of
 * min(L_fwd, K) + min(L_bwd, K).  Lines are found by scanning every base row
 * that can hold a usable sample.
 */
int64_t orc_count_evals(int rows, int cols, int n, double step, double max_range)
{
    int64_t E = 0;
    for (int k = 0; k < n; ++k) {
        orc_dir d;
        if (orc_direction(n, k, rows, cols, step, max_range, &d)) return -1;
        for (int64_t b = -d.D - 1; b <= d.H; ++b) {
            int64_t lo, hi;
            if (orc_line_range(n, k, rows, cols, b, &lo, &hi)) return -1;
            int64_t L = hi - lo + 1;
            E += 2 * sum_min(L, d.K);
        }
    }
    return E;
}

/*
 * The singular viewshed by its definition (Alg. 1-3), without the skewed
 * layout's virtual POVs: the POV is the cell itself, lifted by h0, and each
 * direction's line of sight passes through the cell centre.  Along the view's
 * walk axis the line meets column j at row i + (j - j0) * t, sampled the way
 * Alg. 6 samples (integer part and 32-bit fraction of the fixed-point offset,
 * linear blend of the two rows it falls between, usable iff both rows lie in
 * the DEM).  Each direction adds g * (cv_fwd + cv_bwd) with the walks of
 * Alg. 2 / Alg. 8 read as in walk64; the area is scaled as in Alg. 1.  This is
 * the reference the sDEM discretisation (virtual POVs on lines through whole
 * rows) is compared with, the way section 5 compares sDEM with TVS.
 */
static inline void direct_pos(const orc_dir* d, int64_t i, int64_t j0, int64_t j, int64_t* a, uint32_t* fr)
{
    /* y = (j - j0) * t in 32.32 fixed point; |y| < 2^47.  floor(y / 2^32) and
     * its remainder, for either sign of y. */
    int64_t y = (j - j0) * (int64_t)d->t_fx;
    int64_t q = y >= 0 ? y / (int64_t)4294967296LL : -((-y + 4294967295LL) / (int64_t)4294967296LL);
    *a = i + q;
    *fr = (uint32_t)(y - q * (int64_t)4294967296LL);
}

static inline int direct_ok(const orc_dir* d, int64_t i, int64_t j0, int64_t j)
{
    if (j < 0 || j >= d->W) return 0;
    int64_t a; uint32_t fr;
    direct_pos(d, i, j0, j, &a, &fr);
    if (a < 0) return 0;
    return fr == 0 ? (a <= d->H - 1) : (a + 1 <= d->H - 1);
}

static double direct_walk(const orc_ctx* c, const orc_dir* d, int64_t i, int64_t j0, int dir)
{
    int vis = 1;
    int64_t open = 0, last = 0, cv = 0;
    double h64 = (double)view_at(c->dem, c->cols, d, i, j0) + c->h0;
    float h32 = view_at(c->dem, c->cols, d, i, j0) + (float)c->h0;
    double maxth = -INFINITY;
    float maxth32 = -INFINITY;
    for (int64_t dd = 1; dd <= d->K; ++dd) {
        int64_t j = j0 + dir * dd;
        if (!direct_ok(d, i, j0, j)) break;
        int64_t a; uint32_t fr;
        direct_pos(d, i, j0, j, &a, &fr);
        int above;
        if (c->prec == 64) {
            double z = (double)view_at(c->dem, c->cols, d, a, j);
            if (fr != 0) {
                double r = (double)fr / TWO32;
                z = (1.0 - r) * z + r * (double)view_at(c->dem, c->cols, d, a + 1, j);
            }
            double th = (z - h64) / (double)dd;
            above = th > maxth;
            if (th > maxth) maxth = th;
        } else {
            float z = view_at(c->dem, c->cols, d, a, j);
            if (fr != 0) {
                float r = (float)fr * 0x1p-32f;
                float pa = (1.0f - r) * z;
                float pb = r * view_at(c->dem, c->cols, d, a + 1, j);
                z = pa + pb;
            }
            float diff = z - h32;
            float th = diff * c->rcp[dd];
            above = th > maxth32;
            if (th > maxth32) maxth32 = th;
        }
        if (above && !vis) open = dd;
        if (!above && vis) cv += dd * dd - open * open;
        vis = above;
        last = dd;
    }
    if (vis) cv += last * last - open * open;
    return (double)cv;
}

int orc_direct_viewshed(const float* dem, int rows, int cols, double step, double h0, int n,
                        double max_range, int prec, const int64_t* idx, int64_t count, double* out)
{
    orc_ctx c;
    int rc = ctx_init(&c, dem, rows, cols, step, h0, n, max_range, prec);
    if (rc) return rc;
    if (!idx || !out || count < 0) { ctx_free(&c); return ORC_ERR_ARG; }
    for (int64_t q = 0; q < count; ++q)
        if (idx[q] < 0 || idx[q] >= (int64_t)rows * cols) { ctx_free(&c); return ORC_ERR_ARG; }
    double scale = pappus_scale(n, step);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < count; ++q) {
        int64_t iD = idx[q] / cols, jD = idx[q] % cols;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) {
            const orc_dir* d = &c.dirs[k];
            int64_t i, j;
            to_view(d, iD, jD, &i, &j);
            acc += d->g * (direct_walk(&c, d, i, j, +1) + direct_walk(&c, d, i, j, -1));
        }
        out[q] = scale * acc;
    }
    ctx_free(&c);
    return ORC_OK;
}

/*
 * Visibility map (the boolean result of a singular viewshed, section 1; for
 * several POVs, how many of them see each cell: a multiple viewshed).  Reading
 * (the paper gives no cell rule): the 2n half-lines of Alg. 1 split the plane
 * into sectors of width pi/n around their axes theta = k' pi/n, k' = 0..2n-1
 * (k' >= n is the backward half of direction k' - n; in the D4 views that
 * mirror the DEM, walking +j of the view goes along k' + n).  A cell belongs to the
 * sector whose axis is nearest to the direction from the POV, with
 * q = atan2(di, dj) * n / pi and k' = floor(q + 1/2) mod 2n (di south, dj east,
 * in double precision).  Within the sector, the cell is visible iff the
 * sample of the half-line through the POV cell (as in orc_direct_viewshed) at
 * the cell's walk-axis column is visible (its slope strictly above every
 * earlier one on the half-line); cells past the line's usable samples or past
 * the walk limit are not visible, and the POV's own cell is.  count[c] (int32,
 * rows*cols, accumulated) gains one for each POV that sees cell c.
 */
static void half_line_flags(const orc_ctx* c, const orc_dir* d, int64_t i, int64_t j0, int dir,
                            unsigned char* vis, int64_t cap)
{
    double h64 = (double)view_at(c->dem, c->cols, d, i, j0) + c->h0;
    float h32 = view_at(c->dem, c->cols, d, i, j0) + (float)c->h0;
    double maxth = -INFINITY;
    float maxth32 = -INFINITY;
    for (int64_t dd = 1; dd <= d->K && dd < cap; ++dd) {
        int64_t j = j0 + dir * dd;
        if (!direct_ok(d, i, j0, j)) break;
        int64_t a; uint32_t fr;
        direct_pos(d, i, j0, j, &a, &fr);
        if (c->prec == 64) {
            double z = (double)view_at(c->dem, c->cols, d, a, j);
            if (fr != 0) {
                double r = (double)fr / TWO32;
                z = (1.0 - r) * z + r * (double)view_at(c->dem, c->cols, d, a + 1, j);
            }
            double th = (z - h64) / (double)dd;
            vis[dd] = th > maxth;
            if (th > maxth) maxth = th;
        } else {
            float z = view_at(c->dem, c->cols, d, a, j);
            if (fr != 0) {
                float r = (float)fr * 0x1p-32f;
                float pa = (1.0f - r) * z;
                float pb = r * view_at(c->dem, c->cols, d, a + 1, j);
                z = pa + pb;
            }
            float diff = z - h32;
            float th = diff * c->rcp[dd];
            vis[dd] = th > maxth32;
            if (th > maxth32) maxth32 = th;
        }
    }
}

int orc_visibility_map(const float* dem, int rows, int cols, double step, double h0, int n, double max_range,
                       int prec, const int32_t* pov_ij, int npov, int32_t* count)
{
    orc_ctx c;
    int rc = ctx_init(&c, dem, rows, cols, step, h0, n, max_range, prec);
    if (rc) return rc;
    if (!pov_ij || !count || npov < 1) { ctx_free(&c); return ORC_ERR_ARG; }
    for (int q = 0; q < npov; ++q)
        if (pov_ij[2 * q] < 0 || pov_ij[2 * q] >= rows || pov_ij[2 * q + 1] < 0 || pov_ij[2 * q + 1] >= cols) {
            ctx_free(&c);
            return ORC_ERR_ARG;
        }
    int64_t cap = (rows > cols ? rows : cols) + 1;
    unsigned char* vis = (unsigned char*)calloc((size_t)(2 * n) * (size_t)cap, 1);
    if (!vis) { ctx_free(&c); return ORC_ERR_OOM; }
    for (int q = 0; q < npov; ++q) {
        int64_t i0 = pov_ij[2 * q], jj0 = pov_ij[2 * q + 1];
        memset(vis, 0, (size_t)(2 * n) * (size_t)cap);
        for (int k = 0; k < n; ++k) {
            int64_t i, j;
            to_view(&c.dirs[k], i0, jj0, &i, &j);
            /* slot k: the walk along +j of the view, slot n + k: along -j */
            half_line_flags(&c, &c.dirs[k], i, j, +1, vis + (size_t)k * cap, cap);
            half_line_flags(&c, &c.dirs[k], i, j, -1, vis + (size_t)(n + k) * cap, cap);
        }
        for (int64_t iD = 0; iD < rows; ++iD)
            for (int64_t jD = 0; jD < cols; ++jD) {
                int seen;
                if (iD == i0 && jD == jj0) {
                    seen = 1;
                } else {
                    double qq = atan2((double)(iD - i0), (double)(jD - jj0)) * (double)n / M_PI;
                    int64_t kp = (int64_t)floor(qq + 0.5);
                    kp = ((kp % (2 * n)) + 2 * n) % (2 * n);
                    int k = (int)(kp % n);
                    /* +j of the view points along theta_k in views 0 and 1 (identity,
                     * transpose) and along theta_k + pi in views 2 and 3 (mirrored) */
                    int plus = (c.dirs[k].frame <= 1) == (kp < n);
                    int64_t iv, jv, iv0, jv0;
                    to_view(&c.dirs[k], iD, jD, &iv, &jv);
                    to_view(&c.dirs[k], i0, jj0, &iv0, &jv0);
                    int64_t dd = plus ? jv - jv0 : jv0 - jv;
                    seen = dd >= 1 && dd < cap && vis[(size_t)(plus ? k : n + k) * cap + dd];
                }
                count[iD * cols + jD] += seen;
            }
    }
    free(vis);
    ctx_free(&c);
    return ORC_OK;
}

int orc_abi_version(void) { return 1; }
