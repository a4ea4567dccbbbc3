/*
 * vd_oracle.c -- plain CPU oracle for discrete Voronoi diagrams, JFA and dJFA
 * ("GPU Voronoi Diagrams for Random Moving Seeds", Stevenson-Regla & Navarro).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library: only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or helper with the CUDA
 * path, and the product path never calls it.
 *
 * Everything is written for clarity, not speed: one pixel at a time, the steps
 * in the paper's order.  The only concession to size is an OpenMP "parallel
 * for" over rows of the per-pixel loops, which does not change any result
 * (every pixel is computed independently from read-only inputs).
 *
 * Conventions (readings of the paper, shared with the CUDA side by definition
 * only, never by code):
 *   - maps are row-major int32, w columns by h rows, pixel (x, y) at y*w + x;
 *   - seeds are int32 (x, y) pairs, seed k at xy[2k], xy[2k+1];
 *   - label -1 means "no seed yet";
 *   - Euclidean distance is compared squared, in exact integers; Manhattan
 *     distance is |dx| + |dy|;
 *   - among equal distances the lowest seed index wins (Section III's
 *     closer-seed-wins comparison made a total order);
 *   - a neighbour position outside the grid is skipped;
 *   - each jump pass reads one map and writes another (a gather over the
 *     symmetric neighbourhood, which is what the scatter of Algorithm 1
 *     computes once the order of its writes no longer matters).
 *
 * Parity status: every function below is pinned by a test that does not
 * re-type its formula (brute force, library distance transforms, closed
 * forms, invariants, the worked example of Section III).  The seed update
 * and the repair frame follow a rule of this library's own (the paper leaves
 * insertion and removal to future work): they are pinned by invariants and
 * by the cases that reduce to brute force, not by anything the paper prints.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_METRIC_EUCLID 0
#define ORC_METRIC_MANHATTAN 1
#define ORC_NB_MOORE 0
#define ORC_NB_VON_NEUMANN 1

/* ------------------------------------------------------------------------ */
/* threads                                                                   */
/* ------------------------------------------------------------------------ */

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* distance (Section II, d; Section V-C for the Manhattan variant)           */
/* ------------------------------------------------------------------------ */

static int64_t orc_dist(int64_t sx, int64_t sy, int64_t px, int64_t py, int metric) {
    int64_t dx = sx - px, dy = sy - py;
    if (metric == ORC_METRIC_MANHATTAN) {
        return (dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy);
    }
    return dx * dx + dy * dy;
}

int64_t orc_distance(int32_t sx, int32_t sy, int32_t px, int32_t py, int metric) {
    return orc_dist(sx, sy, px, py, metric);
}

/* ------------------------------------------------------------------------ */
/* schedules: Eq. 2 (JFA) and Eq. 3-4 (dJFA)                                  */
/* ------------------------------------------------------------------------ */

/* ceil(log2(v)) for an integer v >= 1. */
static int orc_ceil_log2(int64_t v) {
    int e = 0;
    while (((int64_t)1 << e) < v) e++;
    return e;
}

/*
 * Eq. 2: k_1 = 2^(ceil(log2 N) - 1) with N the grid side (N = max(w, h) for a
 * rectangle).  For N = 1 the formula gives 1/2, below the last step length
 * 1, so no pass runs; 0 is returned for that case.
 */
int32_t orc_jfa_first_step(int32_t w, int32_t h) {
    int32_t n = w > h ? w : h;
    int e = orc_ceil_log2(n);
    if (e == 0) return 0;
    return (int32_t)1 << (e - 1);
}

/*
 * Eq. 3-4: delta_1 = 2^ceil(log2(max(2 L_avg, d_max))), L_avg = sqrt(w h / s).
 * ceil(log2 max(a, b)) = max(ceil(log2 a), ceil(log2 b)); for a = 2 L_avg the
 * exponent e is the least integer with 2^e >= 2 sqrt(w h / s), i.e. with
 * 4^e * s >= 4 w h, which is decided here in exact integers (no floating log).
 * e may be negative for very dense seeds; d_max = 0 contributes nothing.
 * Returns the exponent; the caller turns it into a step length.
 */
static int orc_djfa_exponent(int32_t w, int32_t h, int64_t s, int32_t d_max) {
    /* no seed at all: L_avg is unbounded, so the cap (JFA's k_1) decides */
    if (s <= 0) return 62;
    /* e_L: least integer e with 4^e * s >= 4 w h. */
    int64_t target = 4 * (int64_t)w * (int64_t)h;
    int e_l;
    if (s >= target) {
        /* e <= 0: find the least e (going down) with s >= target * 4^(-e). */
        e_l = 0;
        while (s >= target * ((int64_t)1 << (2 * (-(e_l - 1)))) && e_l > -30) e_l--;
    } else {
        e_l = 0;
        while ((((int64_t)1 << (2 * e_l)) * s) < target) e_l++;
    }
    int e = e_l;
    if (d_max > 0) {
        int e_d = orc_ceil_log2(d_max);
        if (e_d > e) e = e_d;
    }
    return e;
}

/* delta_1 of Eq. 4 without the cap; 0 when the exponent is negative. */
int64_t orc_djfa_first_step_uncapped(int32_t w, int32_t h, int64_t s, int32_t d_max) {
    int e = orc_djfa_exponent(w, h, s, d_max);
    if (e < 0) return 0;
    return (int64_t)1 << e;
}

/*
 * delta_1 capped at JFA's k_1: by Section V-A, sparse seeds make dJFA fall
 * back to JFA's cost at worst, and Algorithm 1 derives k_m from the diagram
 * before its loop; k_m is read as that cap.
 */
int32_t orc_djfa_first_step(int32_t w, int32_t h, int64_t s, int32_t d_max) {
    int64_t d1 = orc_djfa_first_step_uncapped(w, h, s, d_max);
    int32_t k1 = orc_jfa_first_step(w, h);
    if (d1 > k1) d1 = k1;
    return (int32_t)d1;
}

/*
 * Writes the pass list of one frame: step lengths first, first/2, ..., 1
 * (log2(first) + 1 passes, Section III and Eq. 4), then `extra` more passes
 * (JFA+1 appends k = 1; JFA+2 appends k = 2 then k = 1; Section III), all
 * Moore except the first `vn_waves` which use the Von Neumann neighbourhood
 * (Section V-B).  Returns the number of passes written (at most `cap`).
 */
static int orc_fill_schedule(int32_t first, int vn_waves, int extra,
                             int32_t* ks, int32_t* nbs, int cap) {
    int n = 0;
    for (int32_t k = first; k >= 1; k /= 2) {
        if (n < cap) {
            ks[n] = k;
            nbs[n] = (n < vn_waves) ? ORC_NB_VON_NEUMANN : ORC_NB_MOORE;
        }
        n++;
    }
    for (int e = extra; e >= 1; e--) {
        if (n < cap) {
            ks[n] = (int32_t)1 << (e - 1);
            nbs[n] = ORC_NB_MOORE;
        }
        n++;
    }
    return n;
}

int orc_jfa_schedule(int32_t w, int32_t h, int extra, int32_t* ks, int32_t* nbs, int cap) {
    return orc_fill_schedule(orc_jfa_first_step(w, h), 0, extra, ks, nbs, cap);
}

int orc_djfa_schedule(int32_t w, int32_t h, int64_t s, int32_t d_max, int vn_waves,
                      int extra, int32_t* ks, int32_t* nbs, int cap) {
    return orc_fill_schedule(orc_djfa_first_step(w, h, s, d_max), vn_waves, extra, ks, nbs, cap);
}

/* ------------------------------------------------------------------------ */
/* the exact diagram, Eq. 1                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Brute force over all seeds for every pixel: label = the lowest k that
 * attains min_k d(x, P_k) (Eq. 1 with the lowest-index reading of "<="),
 * dist = that minimum.  Either output may be NULL.
 */
void orc_exact_brute(int32_t w, int32_t h, int64_t s, const int32_t* xy, int metric,
                     int32_t* label, int32_t* dist) {
#pragma omp parallel for schedule(static)
    for (int32_t y = 0; y < h; y++) {
        for (int32_t x = 0; x < w; x++) {
            int64_t best_d = -1;
            int64_t best_k = -1;
            for (int64_t k = 0; k < s; k++) {
                int64_t d = orc_dist(xy[2 * k], xy[2 * k + 1], x, y, metric);
                if (best_k < 0 || d < best_d) {
                    best_d = d;
                    best_k = k;
                }
            }
            int64_t i = (int64_t)y * w + x;
            if (label) label[i] = (int32_t)best_k;
            if (dist) dist[i] = (int32_t)best_d;
        }
    }
}

/*
 * Exact distance map D*(x) = min_k d(x, P_k) without the O(pixels * seeds)
 * cost, for grids where brute force is too slow.
 *
 * Euclidean: the separable squared distance transform of Felzenszwalb and
 * Huttenlocher ("Distance Transforms of Sampled Functions", Theory of
 * Computing 8, 2012): a 1D lower envelope of parabolas down every column of
 * the seed indicator (0 on a seed pixel, infinity elsewhere), then along every
 * row of that result.  The envelope breakpoints are rationals compared by
 * exact integer cross-multiplication.
 *
 * Manhattan: the L1 transform is separable too, and in 1D it is a forward and
 * a backward sweep d[i] = min(d[i], d[i -/+ 1] + 1).
 *
 * Pixels when s = 0 get INT32_MAX.
 */
#define ORC_INF INT64_MAX

/* 1D squared transform of f (length n, ORC_INF = no sample) into out. */
static void orc_dt1d_sq(const int64_t* f, int64_t n, int64_t* out, int64_t* v,
                        int64_t* zn, int64_t* zd) {
    /* v[j]: abscissa of the j-th parabola of the lower envelope; its region
     * starts at z[j] = zn[j]/zd[j] (zd > 0); z[0] = -inf, z[m] = +inf. */
    int64_t m = -1;
    for (int64_t q = 0; q < n; q++) {
        if (f[q] == ORC_INF) continue;
        if (m < 0) {
            m = 0;
            v[0] = q;
            continue;
        }
        for (;;) {
            int64_t p = v[m];
            /* intersection of the parabolas rooted at p and q:
             * s = ((f[q] + q^2) - (f[p] + p^2)) / (2q - 2p) */
            int64_t num = (f[q] + q * q) - (f[p] + p * p);
            int64_t den = 2 * q - 2 * p;
            /* pop while s <= z[m] (z[0] is -inf, never popped) */
            if (m > 0 && num * zd[m] <= zn[m] * den) {
                m--;
                continue;
            }
            m++;
            v[m] = q;
            zn[m] = num;
            zd[m] = den;
            break;
        }
    }
    if (m < 0) {
        for (int64_t i = 0; i < n; i++) out[i] = ORC_INF;
        return;
    }
    int64_t j = 0;
    for (int64_t i = 0; i < n; i++) {
        /* advance while the next region starts at or before i: z[j+1] <= i */
        while (j < m && zn[j + 1] <= i * zd[j + 1]) j++;
        int64_t d = i - v[j];
        out[i] = d * d + f[v[j]];
    }
}

/* 1D Manhattan transform. */
static void orc_dt1d_l1(const int64_t* f, int64_t n, int64_t* out) {
    for (int64_t i = 0; i < n; i++) out[i] = f[i];
    for (int64_t i = 1; i < n; i++)
        if (out[i - 1] != ORC_INF && out[i - 1] + 1 < out[i]) out[i] = out[i - 1] + 1;
    for (int64_t i = n - 2; i >= 0; i--)
        if (out[i + 1] != ORC_INF && out[i + 1] + 1 < out[i]) out[i] = out[i + 1] + 1;
}

void orc_exact_dist_edt(int32_t w, int32_t h, int64_t s, const int32_t* xy, int metric,
                        int32_t* dist) {
    int64_t npx = (int64_t)w * h;
    int64_t* g = (int64_t*)malloc(sizeof(int64_t) * npx);
    for (int64_t i = 0; i < npx; i++) g[i] = ORC_INF;
    for (int64_t k = 0; k < s; k++) g[(int64_t)xy[2 * k + 1] * w + xy[2 * k]] = 0;
    int64_t len = w > h ? w : h;

    /* columns */
#pragma omp parallel
    {
        int64_t* f = (int64_t*)malloc(sizeof(int64_t) * len);
        int64_t* o = (int64_t*)malloc(sizeof(int64_t) * len);
        int64_t* v = (int64_t*)malloc(sizeof(int64_t) * len);
        int64_t* zn = (int64_t*)malloc(sizeof(int64_t) * (len + 1));
        int64_t* zd = (int64_t*)malloc(sizeof(int64_t) * (len + 1));
#pragma omp for schedule(static)
        for (int32_t x = 0; x < w; x++) {
            for (int32_t y = 0; y < h; y++) f[y] = g[(int64_t)y * w + x];
            if (metric == ORC_METRIC_MANHATTAN) orc_dt1d_l1(f, h, o);
            else orc_dt1d_sq(f, h, o, v, zn, zd);
            for (int32_t y = 0; y < h; y++) g[(int64_t)y * w + x] = o[y];
        }
        /* rows (the implicit barrier of "omp for" separates the two sweeps) */
#pragma omp for schedule(static)
        for (int32_t y = 0; y < h; y++) {
            for (int32_t x = 0; x < w; x++) f[x] = g[(int64_t)y * w + x];
            if (metric == ORC_METRIC_MANHATTAN) orc_dt1d_l1(f, w, o);
            else orc_dt1d_sq(f, w, o, v, zn, zd);
            for (int32_t x = 0; x < w; x++) {
                int64_t d = o[x];
                dist[(int64_t)y * w + x] = d == ORC_INF ? INT32_MAX : (int32_t)d;
            }
        }
        free(f);
        free(o);
        free(v);
        free(zn);
        free(zd);
    }
    free(g);
}

/* ------------------------------------------------------------------------ */
/* the moving seeds (Sections IV and V-A, Algorithm 1 SimulateParticles)      */
/* ------------------------------------------------------------------------ */

/* Each seed moves by its given integer displacement, clamped to the grid. */
void orc_move(int32_t w, int32_t h, int64_t s, int32_t* xy, const int32_t* dxy) {
    for (int64_t k = 0; k < s; k++) {
        int64_t x = (int64_t)xy[2 * k] + dxy[2 * k];
        int64_t y = (int64_t)xy[2 * k + 1] + dxy[2 * k + 1];
        if (x < 0) x = 0;
        if (x > w - 1) x = w - 1;
        if (y < 0) y = 0;
        if (y > h - 1) y = h - 1;
        xy[2 * k] = (int32_t)x;
        xy[2 * k + 1] = (int32_t)y;
    }
}

/*
 * SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the n-th output (n = 0, 1, ...) of the
 * generator started at state `seed` is mix(seed + (n + 1) * gamma) with the
 * published golden-ratio gamma and the variant-13 finaliser.
 */
uint64_t orc_splitmix64(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * Uniform integer in [0, m) from a 64-bit draw: Lemire's multiply-shift
 * ("Fast random integer generation in an interval", 2019) on the high 32 bits
 * (the small bias of skipping the rejection step is accepted).
 */
static uint32_t orc_bounded(uint64_t draw, uint32_t m) {
    return (uint32_t)(((draw >> 32) * (uint64_t)m) >> 32);
}

/*
 * Displacement drawn for (stream, step, seed index k, axis a) with maximum
 * |move| D per axis: stream key = splitmix64(rng_seed, stream); draw =
 * splitmix64(key, step * 2^33 + 2k + a); displacement = bounded(draw, 2D+1) - D.
 */
int32_t orc_rng_displacement(uint64_t rng_seed, uint64_t stream, uint64_t step, uint64_t k,
                             int axis, int32_t max_disp) {
    uint64_t key = orc_splitmix64(rng_seed, stream);
    uint64_t n = (step << 33) + 2 * k + (uint64_t)axis;
    return (int32_t)orc_bounded(orc_splitmix64(key, n), (uint32_t)(2 * max_disp + 1)) - max_disp;
}

void orc_move_rng(int32_t w, int32_t h, int64_t s, int32_t* xy, int32_t max_disp,
                  uint64_t rng_seed, uint64_t stream, uint64_t step) {
    for (int64_t k = 0; k < s; k++) {
        int32_t d[2];
        d[0] = orc_rng_displacement(rng_seed, stream, step, (uint64_t)k, 0, max_disp);
        d[1] = orc_rng_displacement(rng_seed, stream, step, (uint64_t)k, 1, max_disp);
        orc_move(w, h, 1, xy + 2 * k, d);
    }
}

/* ------------------------------------------------------------------------ */
/* JFA / dJFA                                                                */
/* ------------------------------------------------------------------------ */

void orc_fill(int32_t w, int32_t h, int32_t* label, int32_t value) {
    int64_t n = (int64_t)w * h;
    for (int64_t i = 0; i < n; i++) label[i] = value;
}

/*
 * Stamp: every seed pixel gets the lowest index among the seeds standing on
 * it, overwriting what the map held there (the flood starts from the seeds,
 * Section III; dJFA re-stamps the moved seeds onto the previous frame's map,
 * Section V).  Writing the indices from the highest down makes the last
 * write the lowest.
 */
void orc_stamp(int32_t w, int32_t h, int64_t s, const int32_t* xy, int32_t* label) {
    (void)h;
    for (int64_t k = s - 1; k >= 0; k--) {
        label[(int64_t)xy[2 * k + 1] * w + xy[2 * k]] = (int32_t)k;
    }
}

/*
 * One jump pass with step k (Table I for the Moore neighbourhood, Section
 * IV-B for Von Neumann): for every pixel q the candidates are q itself and
 * its neighbours at offset k; an out-of-grid neighbour and a label of -1 are
 * skipped; the winner is the candidate seed at the smallest distance from q,
 * the lowest index among equal distances.  Reads src, writes dst.
 */
void orc_pass(int32_t w, int32_t h, const int32_t* xy, const int32_t* src, int32_t* dst,
              int32_t k, int nb, int metric) {
    /* Table I lists the 8 Moore neighbours; Von Neumann keeps the 4 axial. */
    static const int moore[8][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 1},
                                    {-1, 0}, {-1, -1}, {0, -1}, {1, -1}};
#pragma omp parallel for schedule(static)
    for (int32_t y = 0; y < h; y++) {
        for (int32_t x = 0; x < w; x++) {
            int64_t qi = (int64_t)y * w + x;
            int32_t best = src[qi];
            int64_t best_d = best >= 0 ? orc_dist(xy[2 * best], xy[2 * best + 1], x, y, metric) : 0;
            for (int j = 0; j < 8; j++) {
                int ox = moore[j][0], oy = moore[j][1];
                if (nb == ORC_NB_VON_NEUMANN && ox != 0 && oy != 0) continue;
                int64_t nx = (int64_t)x + (int64_t)ox * k;
                int64_t ny = (int64_t)y + (int64_t)oy * k;
                if (nx < 0 || nx >= w || ny < 0 || ny >= h) continue;
                int32_t c = src[ny * w + nx];
                if (c < 0) continue;
                int64_t d = orc_dist(xy[2 * c], xy[2 * c + 1], x, y, metric);
                if (best < 0 || d < best_d || (d == best_d && c < best)) {
                    best = c;
                    best_d = d;
                }
            }
            dst[qi] = best;
        }
    }
}

/* Runs the passes of a schedule on `label` (in/out) with a scratch map. */
static void orc_run_passes(int32_t w, int32_t h, const int32_t* xy, int32_t* label,
                           const int32_t* ks, const int32_t* nbs, int n, int metric) {
    int64_t npx = (int64_t)w * h;
    int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (npx > 0 ? npx : 1));
    int32_t* a = label;
    int32_t* b = tmp;
    for (int i = 0; i < n; i++) {
        orc_pass(w, h, xy, a, b, ks[i], nbs[i], metric);
        int32_t* t = a;
        a = b;
        b = t;
    }
    if (a != label) memcpy(label, a, sizeof(int32_t) * npx);
    free(tmp);
}

/*
 * JFA from scratch (Section III): an empty map, the seeds stamped, then the
 * passes k_1, k_1/2, ..., 1 of Eq. 2 with the Moore neighbourhood, plus
 * `extra` JFA+1 / JFA+2 passes.
 */
void orc_jfa(int32_t w, int32_t h, int64_t s, const int32_t* xy, int extra, int metric,
             int32_t* label) {
    int32_t ks[80], nbs[80];
    int n = orc_jfa_schedule(w, h, extra, ks, nbs, 80);
    orc_fill(w, h, label, -1);
    orc_stamp(w, h, s, xy, label);
    orc_run_passes(w, h, xy, label, ks, nbs, n, metric);
}

/*
 * One dJFA step (Section V, Algorithm 1, after SimulateParticles): the
 * moved seeds are stamped onto the previous frame's map held in `label`,
 * then the passes delta_1, ..., 1 of Eq. 4 run, the first `vn_waves` with
 * the Von Neumann neighbourhood and the rest Moore, plus `extra` passes.
 */
void orc_djfa_step(int32_t w, int32_t h, int64_t s, const int32_t* xy, int32_t d_max,
                   int vn_waves, int extra, int metric, int32_t* label) {
    int32_t ks[80], nbs[80];
    int n = orc_djfa_schedule(w, h, s, d_max, vn_waves, extra, ks, nbs, 80);
    orc_stamp(w, h, s, xy, label);
    orc_run_passes(w, h, xy, label, ks, nbs, n, metric);
}

/* ------------------------------------------------------------------------ */
/* seed insertion and removal (Section VII leaves it to future work; the rule */
/* below is this library's reading, pinned by the invariants in the tests)    */
/* ------------------------------------------------------------------------ */

/*
 * Seed update between frames: the seeds listed in `remove` (distinct indices
 * in [0, s)) leave, the survivors keep their order and are renumbered
 * 0 .. s_keep - 1, and the n_add seeds of `add` follow as s_keep, s_keep + 1,
 * ...  The map is relabelled to match: a pixel labelled with a surviving seed
 * takes that seed's new index, a pixel labelled with a removed seed becomes
 * empty (-1).  Writes the new seed array to out_xy and returns its length;
 * returns -1 (and changes nothing) when `remove` holds an index out of range
 * or twice, an added seed lies outside the grid, or no seed would remain.
 */
int64_t orc_update_seeds(int32_t w, int32_t h, int64_t s, const int32_t* xy, int32_t* label,
                         const int32_t* remove, int64_t n_remove, const int32_t* add, int64_t n_add,
                         int32_t* out_xy) {
    if (n_remove < 0 || n_add < 0 || s - n_remove + n_add < 1) return -1;
    for (int64_t j = 0; j < n_add; j++) {
        if (add[2 * j] < 0 || add[2 * j] >= w || add[2 * j + 1] < 0 || add[2 * j + 1] >= h) return -1;
    }
    char* gone = (char*)calloc((size_t)(s > 0 ? s : 1), 1);
    for (int64_t j = 0; j < n_remove; j++) {
        int32_t id = remove[j];
        if (id < 0 || id >= s || gone[id]) {
            free(gone);
            return -1;
        }
        gone[id] = 1;
    }
    /* the survivors' new indices, in their old order */
    int32_t* renum = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s > 0 ? s : 1));
    int64_t kept = 0;
    for (int64_t k = 0; k < s; k++) {
        if (gone[k]) {
            renum[k] = -1;
        } else {
            renum[k] = (int32_t)kept;
            out_xy[2 * kept] = xy[2 * k];
            out_xy[2 * kept + 1] = xy[2 * k + 1];
            kept++;
        }
    }
    for (int64_t j = 0; j < n_add; j++) {
        out_xy[2 * (kept + j)] = add[2 * j];
        out_xy[2 * (kept + j) + 1] = add[2 * j + 1];
    }
    int64_t npx = (int64_t)w * h;
    for (int64_t i = 0; i < npx; i++) {
        if (label[i] >= 0) label[i] = renum[label[i]];
    }
    free(renum);
    free(gone);
    return kept + n_add;
}

/*
 * The frame after a removal: the current seeds are stamped onto the
 * relabelled map and the full JFA schedule (Eq. 2, Moore, plus `extra`
 * passes) runs on it without clearing, so the emptied cells fill from every
 * side whatever their size.
 */
void orc_repair_step(int32_t w, int32_t h, int64_t s, const int32_t* xy, int extra, int metric,
                     int32_t* label) {
    int32_t ks[80], nbs[80];
    int n = orc_jfa_schedule(w, h, extra, ks, nbs, 80);
    orc_stamp(w, h, s, xy, label);
    orc_run_passes(w, h, xy, label, ks, nbs, n, metric);
}

/* ------------------------------------------------------------------------ */
/* similarity (Section VI-A)                                                 */
/* ------------------------------------------------------------------------ */

/*
 * n_match: pixels whose label equals ref_label (the paper's similarity is
 * 100 * n_match / pixels against a full JFA).  n_exact: pixels whose label's
 * seed lies at the exact minimum distance exact_dist (the distance-correct
 * count against Eq. 1).  Either reference may be NULL (its count is then 0).
 */
void orc_similarity(int32_t w, int32_t h, const int32_t* xy, const int32_t* label,
                    const int32_t* exact_dist, const int32_t* ref_label, int metric,
                    uint64_t* n_exact, uint64_t* n_match) {
    uint64_t ne = 0, nm = 0;
#pragma omp parallel for schedule(static) reduction(+ : ne, nm)
    for (int32_t y = 0; y < h; y++) {
        for (int32_t x = 0; x < w; x++) {
            int64_t i = (int64_t)y * w + x;
            int32_t l = label[i];
            if (exact_dist && l >= 0 &&
                orc_dist(xy[2 * l], xy[2 * l + 1], x, y, metric) == exact_dist[i])
                ne++;
            if (ref_label && l == ref_label[i]) nm++;
        }
    }
    *n_exact = ne;
    *n_match = nm;
}
