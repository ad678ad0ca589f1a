/*
 * csg_oracle.c -- the CPU oracle for the causal-set hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load it.  It shares no source,
 * header, table or helper with the CUDA library, and the library never calls it.
 *
 * Everything follows Cunningham & Krioukov, "Causal Set Generator and Action
 * Computer" (arXiv:1709.03013):
 *   - sprinkling into a flat causal diamond          (Sec. 2.1, Fig. 1)
 *   - labelling elements in time order               (Sec. 2.2)
 *   - a dense symmetric 0/1 adjacency matrix         (Sec. 2.2)
 *   - interval abundances by the naive triple loop   (Sec. 4.1, with the
 *     per-thread private histograms of Sec. 4.2)
 *   - the 1+1 BD action S2                           (Eq. s_local)
 *   - the 3+1 BD action S4 = (4/sqrt6)(N-N0+9N1-16N2+8N3)  (Benincasa-Dowker,
 *     cited in Sec. 1.2; the paper prints only the 1+1 form)
 *   - the smeared action S_eps                       (Eq. s_smeared)
 *   - sprinkling into the 1+1 de Sitter slab         (Sec. 5.1)
 *   - the discrete d'Alembertian B phi per element   (Eq. b_local)
 *
 * Readings where the paper is silent (listed in the design notes too):
 *   - RNG: Philox4x64-10 (Salmon et al., SC'11), counter (element, attempt, 0, 0),
 *     key (seed, seq); a 64-bit draw x maps to (x >> 11) * 2^-53 in [0, 1).
 *   - d=2: u, v from the first two words of attempt 0; t = (u+v)/2, x = (v-u)/2;
 *     i < j related iff u_i < u_j and v_i < v_j.
 *   - d=4: attempt a gives (t,x,y,z) = 2*U - 1 from the four words; the first
 *     attempt with |t| + sqrt((x*x + y*y) + z*z) <= 1 is kept, at most 256 tries.
 *     i < j related iff t_j > t_i and dt*dt > (dx*dx + dy*dy) + dz*dz, all in
 *     IEEE double with no fused multiply-add (compile with -ffp-contract=off).
 *   - sort key: (t, u, element) for d=2, (t, element) for d=4.
 *   - the paper's 1-based abundance n_i equals the 0-based N_{i-1} used here
 *     (Sec. 1.2 defines L_i with i-1 interior elements; Alg. 5 counts into c[m+1]).
 *
 * Parity status: every function here is pinned by a test that does not retype
 * its formula (library Philox, closed forms, brute force, graph-library interval
 * counts, 2D dominance counts, invariants); see the oracle tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Geometry codes: 2 = flat 1+1 diamond, 4 = flat 3+1 diamond,
 * ORC_DS2 = 1+1 de Sitter slab of Sec. 5.1 (coordinates eta, theta). */
#define ORC_DS2 3
#define ORC_GEOM_OK(d) ((d) == 2 || (d) == 4 || (d) == ORC_DS2)

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_EREJECT -3

/* ---------------------------------------------------------------- RNG ---- */

/* Philox4x64-10, written from its published definition: ten rounds of two
 * 64x64->128 multiplications with the round keys bumped by Weyl constants. */
static void orc_philox_round(uint64_t c[4], const uint64_t k[2]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    unsigned __int128 p0 = (unsigned __int128)M0 * c[0];
    unsigned __int128 p1 = (unsigned __int128)M1 * c[2];
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t n0 = hi1 ^ c[1] ^ k[0];
    uint64_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint64_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        orc_philox_round(c, k);
        k[0] += 0x9E3779B97F4A7C15ULL;
        k[1] += 0xBB67AE8584CAA73BULL;
    }
    memcpy(out, c, sizeof c);
}

static double orc_unit(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

/* ------------------------------------------------------------ sprinkle ---- */

/* coords is [4][N] doubles, element order (unsorted):
 *   d=2: rows t, x, u, v        d=4: rows t, x, y, z
 * attempts (optional) receives the accepted attempt index per element. */
int orc_sprinkle(int d, int64_t N, uint64_t seed, uint64_t seq, double *coords,
                 int32_t *attempts) {
    if ((d != 2 && d != 4) || N < 0 || (N > 0 && !coords)) return ORC_EINVAL;
    const uint64_t key[2] = {seed, seq};
    int bad = 0;
    for (int64_t e = 0; e < N; ++e) {
        if (d == 2) {
            uint64_t ctr[4] = {(uint64_t)e, 0, 0, 0}, r[4];
            orc_philox4x64_10(ctr, key, r);
            double u = orc_unit(r[0]);
            double v = orc_unit(r[1]);
            coords[0 * N + e] = (u + v) / 2.0;
            coords[1 * N + e] = (v - u) / 2.0;
            coords[2 * N + e] = u;
            coords[3 * N + e] = v;
            if (attempts) attempts[e] = 0;
        } else {
            int a, found = 0;
            for (a = 0; a < 256; ++a) {
                uint64_t ctr[4] = {(uint64_t)e, (uint64_t)a, 0, 0}, r[4];
                orc_philox4x64_10(ctr, key, r);
                double t = 2.0 * orc_unit(r[0]) - 1.0;
                double x = 2.0 * orc_unit(r[1]) - 1.0;
                double y = 2.0 * orc_unit(r[2]) - 1.0;
                double z = 2.0 * orc_unit(r[3]) - 1.0;
                double rr = sqrt((x * x + y * y) + z * z);
                if (fabs(t) + rr <= 1.0) {
                    coords[0 * N + e] = t;
                    coords[1 * N + e] = x;
                    coords[2 * N + e] = y;
                    coords[3 * N + e] = z;
                    found = 1;
                    break;
                }
            }
            if (!found) bad = 1;
            if (attempts) attempts[e] = found ? a : -1;
        }
    }
    return bad ? ORC_EREJECT : ORC_OK;
}

/* 1+1 de Sitter slab (Sec. 5.1): eta in [-eta0, eta0] with density proportional to
 * sec^2(eta), theta uniform in [0, 2 pi).  Inverting the distribution function
 * (tan eta + tan eta0) / (2 tan eta0) gives eta = atan(tan(eta0) (2U - 1)).  Element e
 * uses words 0 and 1 of the Philox block (e, 0, 0, 0); coords rows are eta, theta, 0, 0. */
int orc_sprinkle_desitter(int64_t N, double eta0, uint64_t seed, uint64_t seq, double *coords) {
    if (N < 0 || (N > 0 && !coords) || !(eta0 > 0.0 && eta0 < 1.5707963267948966)) return ORC_EINVAL;
    const uint64_t key[2] = {seed, seq};
    const double t0 = tan(eta0);
    for (int64_t e = 0; e < N; ++e) {
        uint64_t ctr[4] = {(uint64_t)e, 0, 0, 0}, r[4];
        orc_philox4x64_10(ctr, key, r);
        coords[e] = atan(t0 * (2.0 * orc_unit(r[0]) - 1.0));
        coords[N + e] = 6.283185307179586 * orc_unit(r[1]);
        coords[2 * N + e] = 0.0;
        coords[3 * N + e] = 0.0;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- sort ---- */

typedef struct {
    double t, u;
    int64_t e;
} orc_key;

static int orc_key_cmp(const void *pa, const void *pb) {
    const orc_key *a = (const orc_key *)pa, *b = (const orc_key *)pb;
    if (a->t < b->t) return -1;
    if (a->t > b->t) return 1;
    if (a->u < b->u) return -1;
    if (a->u > b->u) return 1;
    return (a->e < b->e) ? -1 : (a->e > b->e);
}

/* Sorts the elements by time (Sec. 2.2) and permutes coords in place.
 * perm[p] receives the sprinkle index of the element now at position p. */
int orc_sort(int d, int64_t N, double *coords, int64_t *perm) {
    if (!ORC_GEOM_OK(d) || N < 0) return ORC_EINVAL;
    if (N == 0) return ORC_OK;
    orc_key *keys = (orc_key *)malloc((size_t)N * sizeof(orc_key));
    double *tmp = (double *)malloc((size_t)N * 4 * sizeof(double));
    if (!keys || !tmp) {
        free(keys);
        free(tmp);
        return ORC_ENOMEM;
    }
    for (int64_t e = 0; e < N; ++e) {
        keys[e].t = coords[e];
        keys[e].u = (d == 2) ? coords[2 * N + e] : 0.0;
        keys[e].e = e;
    }
    qsort(keys, (size_t)N, sizeof(orc_key), orc_key_cmp);
    memcpy(tmp, coords, (size_t)N * 4 * sizeof(double));
    for (int64_t p = 0; p < N; ++p) {
        int64_t e = keys[p].e;
        for (int r = 0; r < 4; ++r) coords[r * N + p] = tmp[r * N + e];
        if (perm) perm[p] = e;
    }
    free(keys);
    free(tmp);
    return ORC_OK;
}

/* ---------------------------------------------------------------- link ---- */

/* Relation between sorted elements i < j (the later one is j). */
static int orc_precedes(int d, int64_t N, const double *c, int64_t i, int64_t j) {
    if (d == ORC_DS2) {
        /* timelike on the cylinder: the shorter angular separation is below |d eta|
         * (Eq. ds_metric: d theta^2 < d eta^2) */
        const double pi = 3.141592653589793;
        double ang = pi - fabs(pi - fabs(c[N + j] - c[N + i]));
        return ang < fabs(c[j] - c[i]);
    }
    if (d == 2) {
        return c[2 * N + i] < c[2 * N + j] && c[3 * N + i] < c[3 * N + j];
    }
    double ti = c[i], tj = c[j];
    if (!(tj > ti)) return 0;
    double dt = tj - ti;
    double dx = c[1 * N + j] - c[1 * N + i];
    double dy = c[2 * N + j] - c[2 * N + i];
    double dz = c[3 * N + j] - c[3 * N + i];
    double s = (dx * dx + dy * dy) + dz * dz;
    return dt * dt > s;
}

/* Symmetric relation of two sorted elements, either order. */
int orc_related(int d, int64_t N, const double *coords, int64_t i, int64_t j) {
    if (i == j) return 0;
    if (i > j) {
        int64_t s = i;
        i = j;
        j = s;
    }
    return orc_precedes(d, N, coords, i, j);
}

/* Dense symmetric adjacency matrix, one byte per entry (Sec. 2.2.2). */
int orc_link(int d, int64_t N, const double *coords, uint8_t *rel, int threads) {
    if (!ORC_GEOM_OK(d) || N < 0 || (N > 0 && (!coords || !rel))) return ORC_EINVAL;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    (void)threads;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
        rel[i * N + i] = 0;
        for (int64_t j = i + 1; j < N; ++j) {
            uint8_t r = (uint8_t)orc_precedes(d, N, coords, i, j);
            rel[i * N + j] = r;
            rel[j * N + i] = r;
        }
    }
    return ORC_OK;
}

/* One row of the adjacency matrix, for sampled checks at sizes where the full
 * N*N matrix is not built. */
int orc_link_row(int d, int64_t N, const double *coords, int64_t i, uint8_t *row) {
    if (!ORC_GEOM_OK(d) || i < 0 || i >= N) return ORC_EINVAL;
    for (int64_t j = 0; j < N; ++j) row[j] = (uint8_t)orc_related(d, N, coords, i, j);
    return ORC_OK;
}

/* Packs the matrix into the library's layout: row i is stride_words 64-bit
 * words, bit k of the row at word k/64, bit k%64, padding bits zero. */
int orc_pack(int64_t N, const uint8_t *rel, int64_t stride_words, uint64_t *words) {
    if (N < 0 || stride_words * 64 < N) return ORC_EINVAL;
    memset(words, 0, (size_t)(N * stride_words) * sizeof(uint64_t));
    for (int64_t i = 0; i < N; ++i)
        for (int64_t k = 0; k < N; ++k)
            if (rel[i * N + k]) words[i * stride_words + k / 64] |= (uint64_t)1 << (k % 64);
    return ORC_OK;
}

/* -------------------------------------------------------------- action ---- */

/* Size of the open interval between sorted elements i < j: the number of k
 * with i < k < j that are in the future of i and in the past of j (Sec. 4.1). */
int64_t orc_interval(int64_t N, const uint8_t *rel, int64_t i, int64_t j) {
    int64_t m = 0;
    for (int64_t k = i + 1; k < j; ++k) m += rel[i * N + k] & rel[k * N + j];
    return m;
}

/* The same count straight from coordinates, with no matrix: O(N) per pair. */
int64_t orc_interval_coords(int d, int64_t N, const double *coords, int64_t i, int64_t j) {
    int64_t m = 0;
    for (int64_t k = i + 1; k < j; ++k)
        m += orc_precedes(d, N, coords, i, k) & orc_precedes(d, N, coords, k, j);
    return m;
}

/* Interval abundances over rows [row_lo, row_hi) (all rows: 0, N).
 *   hist[m] += 1 for every related pair i < j with i in the row range, where
 *   m = |{k : i < k < j, i rel k, k rel j}|; hist has max(N,1) bins (m <= N-2).
 *   R = number of related pairs counted, sum_m = sum of m,
 *   W = sum of (j - i - 1), the candidate bits inspected.
 * The triple loop follows Sec. 4.1; rows are spread over threads with one
 * private histogram each, reduced at the end (Sec. 4.2).  The inner loop reads
 * row j instead of column j, which is the same entry because the matrix is
 * symmetric (Sec. 2.2). */
int orc_action_rows(int64_t N, const uint8_t *rel, int64_t row_lo, int64_t row_hi,
                    uint64_t *hist, uint64_t *R, uint64_t *sum_m, uint64_t *W, int threads) {
    if (N < 0 || row_lo < 0 || row_hi > N || row_lo > row_hi) return ORC_EINVAL;
    int64_t bins = N > 0 ? N : 1;
    memset(hist, 0, (size_t)bins * sizeof(uint64_t));
    uint64_t tR = 0, tS = 0, tW = 0;
#ifdef _OPENMP
    int T = threads > 0 ? threads : omp_get_max_threads();
#else
    int T = 1;
#endif
    (void)threads;
    uint64_t *priv = (uint64_t *)calloc((size_t)T * (size_t)bins, sizeof(uint64_t));
    if (!priv) return ORC_ENOMEM;
#pragma omp parallel num_threads(T) reduction(+ : tR, tS, tW)
    {
#ifdef _OPENMP
        uint64_t *h = priv + (size_t)omp_get_thread_num() * (size_t)bins;
#else
        uint64_t *h = priv;
#endif
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = row_lo; i < row_hi; ++i) {
            const uint8_t *ri = rel + i * N;
            for (int64_t j = i + 1; j < N; ++j) {
                if (!ri[j]) continue;
                const uint8_t *rj = rel + j * N;
                /* m <= N - 2 < 2^31 (the largest interval, Sec. 4.1): a 32-bit count is exact */
                uint32_t m = 0;
                for (int64_t k = i + 1; k < j; ++k) m += ri[k] & rj[k];
                h[m] += 1;
                tR += 1;
                tS += (uint64_t)m;
                tW += (uint64_t)(j - i - 1);
            }
        }
    }
    for (int t = 0; t < T; ++t)
        for (int64_t b = 0; b < bins; ++b) hist[b] += priv[(size_t)t * (size_t)bins + b];
    free(priv);
    *R = tR;
    *sum_m = tS;
    *W = tW;
    return ORC_OK;
}

/* The same abundances for rows [row_lo, row_hi), computed straight from the sorted
 * coordinates with no N*N matrix: for each related pair i < j with i in the range,
 * m counts the k with i < k < j related to both (Sec. 4.1).  O(N^2) per row; used
 * to check sampled rows of sets too large for the matrix. */
int orc_action_rows_coords(int d, int64_t N, const double *coords, int64_t row_lo, int64_t row_hi,
                           uint64_t *hist, uint64_t *R, uint64_t *sum_m, uint64_t *W, int threads) {
    if (!ORC_GEOM_OK(d) || N < 0 || row_lo < 0 || row_hi > N || row_lo > row_hi) return ORC_EINVAL;
    int64_t bins = N > 0 ? N : 1;
    memset(hist, 0, (size_t)bins * sizeof(uint64_t));
    uint64_t tR = 0, tS = 0, tW = 0;
#ifdef _OPENMP
    int T = threads > 0 ? threads : omp_get_max_threads();
#else
    int T = 1;
#endif
    (void)threads;
    uint64_t *priv = (uint64_t *)calloc((size_t)T * (size_t)bins, sizeof(uint64_t));
    uint8_t *fut = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    if (!priv || !fut) {
        free(priv);
        free(fut);
        return ORC_ENOMEM;
    }
    for (int64_t i = row_lo; i < row_hi; ++i) {
        for (int64_t k = 0; k < N; ++k) fut[k] = (uint8_t)(k > i && orc_precedes(d, N, coords, i, k));
#pragma omp parallel num_threads(T) reduction(+ : tR, tS, tW)
        {
#ifdef _OPENMP
            uint64_t *h = priv + (size_t)omp_get_thread_num() * (size_t)bins;
#else
            uint64_t *h = priv;
#endif
#pragma omp for schedule(dynamic, 64)
            for (int64_t j = i + 1; j < N; ++j) {
                if (!fut[j]) continue;
                int64_t m = 0;
                for (int64_t k = i + 1; k < j; ++k)
                    if (fut[k]) m += orc_precedes(d, N, coords, k, j);
                h[m] += 1;
                tR += 1;
                tS += (uint64_t)m;
                tW += (uint64_t)(j - i - 1);
            }
        }
    }
    for (int t = 0; t < T; ++t)
        for (int64_t b = 0; b < bins; ++b) hist[b] += priv[(size_t)t * (size_t)bins + b];
    free(priv);
    free(fut);
    *R = tR;
    *sum_m = tS;
    *W = tW;
    return ORC_OK;
}

int orc_action(int64_t N, const uint8_t *rel, uint64_t *hist, uint64_t *R, uint64_t *sum_m,
               uint64_t *W, int threads) {
    return orc_action_rows(N, rel, 0, N, hist, R, sum_m, W, threads);
}

/* ------------------------------------------------------------ finalize ---- */

/* d=2: combo = N - 2N0 + 4N1 - 2N2 and S = 2*combo        (Eq. s_local)
 * d=4: combo = N - N0 + 9N1 - 16N2 + 8N3, S = (4/sqrt6)*combo. */
int orc_finalize(int d, int64_t N, const uint64_t Nk[4], int64_t *combo, double *S) {
    if (d == 2) {
        int64_t c = N - 2 * (int64_t)Nk[0] + 4 * (int64_t)Nk[1] - 2 * (int64_t)Nk[2];
        *combo = c;
        *S = 2.0 * (double)c;
        return ORC_OK;
    }
    if (d == 4) {
        int64_t c = N - (int64_t)Nk[0] + 9 * (int64_t)Nk[1] - 16 * (int64_t)Nk[2] +
                    8 * (int64_t)Nk[3];
        *combo = c;
        *S = (4.0 / sqrt(6.0)) * (double)c;
        return ORC_OK;
    }
    return ORC_EINVAL;
}

/* Smeared (non-local) action of Eq. s_smeared from the full 0-based histogram
 * hist[0..N-2] (hist[m] = pairs whose interval holds m elements, so the paper's
 * 1-based n_i is hist[i-1]):
 *   S_eps = 2 eps [ N - 2 eps sum_{i=1}^{N-1} n_i f2(i-1, eps) ],
 *   f2(i, eps) = (1-eps)^i [1 - 2 eps i/(1-eps) + eps^2 i (i-1) / (2 (1-eps)^2)],
 * for 0 < eps < 1.  The sum runs in increasing i. */
double orc_smeared(int64_t N, const uint64_t *hist, double eps) {
    double acc = 0.0;
    for (int64_t i = 1; i <= N - 1; ++i) {
        const uint64_t n_i = hist[i - 1];
        if (n_i == 0) continue;
        const double a = (double)(i - 1);
        const double q = 1.0 - eps;
        const double f2 = pow(q, a) * (1.0 - 2.0 * eps * a / q + eps * eps * a * (a - 1.0) / (2.0 * q * q));
        acc += (double)n_i * f2;
    }
    return 2.0 * eps * ((double)N - 2.0 * eps * acc);
}

/* ------------------------------------------------------- d'Alembertian ---- */

/* Discrete d'Alembertian of Eq. b_local (Sec. 1.2), 1+1 dimensions:
 *   B phi(x) = (2 / l^2) ( -phi(x) + 2 [ sum_{y in L_1} - 2 sum_{y in L_2} + sum_{y in L_3} ] phi(y) ),
 * where L_i is the set of elements y preceding x with exactly i - 1 elements z strictly
 * between them (y < z < x).  rel is the symmetric relation matrix of time-ordered
 * elements, so y precedes x iff y < x and rel[y][x].  For every x the three sums run over
 * y in increasing label order and are combined as printed.  The work is O(N^3). */
int orc_dalembertian(int64_t N, const uint8_t *rel, const double *phi, double l, double *out,
                     int64_t *L123, int threads) {
    if (N < 0 || (N > 0 && (!rel || !phi || !out)) || !(l > 0.0)) return ORC_EINVAL;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t x = 0; x < N; ++x) {
        double s[3] = {0.0, 0.0, 0.0};
        int64_t cnt[3] = {0, 0, 0};
        for (int64_t y = 0; y < x; ++y) {
            if (!rel[y * N + x]) continue;
            int64_t m = 0;
            for (int64_t z = y + 1; z < x; ++z) m += rel[y * N + z] & rel[z * N + x];
            if (m <= 2) {
                s[m] += phi[y];
                cnt[m] += 1;
            }
        }
        out[x] = (2.0 / (l * l)) * (-phi[x] + 2.0 * (s[0] - 2.0 * s[1] + s[2]));
        if (L123)
            for (int k = 0; k < 3; ++k) L123[3 * x + k] = cnt[k];
    }
    return ORC_OK;
}
