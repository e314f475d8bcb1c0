/*
 * Plain CPU oracle for the Cornerstone octree build (Keller et al., PASC'23, arXiv 2307.06345).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU-baseline leg of the
 * benchmark; never by the product library. It shares no code with the CUDA path.
 *
 * Compile with -O2 -ffp-contract=off: each floating-point expression below is then evaluated as
 * the written sequence of IEEE-754 double round-to-nearest operations.
 *
 * Loops whose iterations are independent (one particle, leaf or node each; every iteration
 * writes only its own outputs and reads nothing another iteration writes) carry an OpenMP
 * `parallel for`. Each iteration computes exactly what the sequential loop computes, in the same
 * operation order, so results do not depend on the thread count (oracle_set_threads; 1 = the
 * plain sequential program). The sorts qsort contiguous chunks in parallel and merge them; the
 * order they produce is total (distinct (key, index) pairs, distinct node keys), so it is unique.
 */
#include "cstone_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define L ORACLE_L
#define KEY_END (1ULL << (3 * L)) /* 8^L (2^63 at L = 21), one past the last key */

/* Threads of the parallel loops (the machine's cores by default; 1 = sequential). */
void oracle_set_threads(int threads) {
#ifdef _OPENMP
    omp_set_num_threads(threads > 0 ? threads : omp_get_num_procs());
#else
    (void)threads;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sorts n elements of `size` bytes into ascending order under `cmp`, where elements that compare
 * equal are identical, so the result is unique: contiguous chunks are qsorted, one per thread,
 * then merged pairwise. `tmp` holds n elements. */
static void sort_total(void* base, void* tmp, int64_t n, size_t size, int (*cmp)(const void*, const void*)) {
    int chunks = oracle_get_threads();
    if (chunks < 1 || n < 4096) chunks = 1;
    int64_t per = (n + chunks - 1) / chunks;
    char* a = (char*)base;
    char* b = (char*)tmp;
#pragma omp parallel for schedule(static, 1)
    for (int c = 0; c < chunks; ++c) {
        int64_t lo = c * per, hi = lo + per < n ? lo + per : n;
        if (hi > lo) qsort(a + lo * size, (size_t)(hi - lo), size, cmp);
    }
    for (int64_t width = per; width < n; width *= 2) {
        int64_t pairs = (n + 2 * width - 1) / (2 * width);
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t q = 0; q < pairs; ++q) {
            int64_t lo = q * 2 * width;
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) {
                if (cmp(a + i * size, a + j * size) < 0)
                    memcpy(b + (k++) * size, a + (i++) * size, size);
                else
                    memcpy(b + (k++) * size, a + (j++) * size, size);
            }
            if (i < mid) memcpy(b + k * size, a + i * size, (size_t)(mid - i) * size), k += mid - i;
            if (j < hi) memcpy(b + k * size, a + j * size, (size_t)(hi - j) * size);
        }
        char* t = a;
        a = b;
        b = t;
    }
    if (a != (char*)base) memcpy(base, a, (size_t)n * size);
}

/* =====================================================================================
 * Sec. 3: keys. A key of 3L bits is a sequence of L octal digits; digit i selects the octant
 * at division level i. Grid coordinates live in [0, 2^L) per axis.
 * ===================================================================================== */

/* Bounding cube (the paper is silent on normalisation): lo = per-axis minimum, side = the largest
 * per-axis extent (max - min), side = 1 when that extent is 0 or there are no points. Min and max
 * are exact; the extent is one rounded subtraction per axis. */
int oracle_bounding_cube(const double* x, const double* y, const double* z, int64_t n, double box[4]) {
    if (n < 0) return ORACLE_E_ARG;
    if (n == 0) {
        box[0] = box[1] = box[2] = 0.0;
        box[3] = 1.0;
        return ORACLE_OK;
    }
    const double* c[3] = {x, y, z};
    double side = 0.0;
    for (int d = 0; d < 3; ++d) {
        double lo = c[d][0], hi = c[d][0];
        for (int64_t i = 1; i < n; ++i) {
            if (c[d][i] < lo) lo = c[d][i];
            if (c[d][i] > hi) hi = c[d][i];
        }
        box[d] = lo;
        double ext = hi - lo;
        if (ext > side) side = ext;
    }
    box[3] = (side > 0.0) ? side : 1.0;
    return ORACLE_OK;
}

/* Sec. 6: the cube of a point set spread over several processes, from the per-axis bounds
 * {min x, min y, min z, max x, max y, max z} reduced over the processes (the minima of the minima,
 * the maxima of the maxima). Same arithmetic as oracle_bounding_cube: lo = minima, side = the
 * largest extent, 1 when that extent is 0 or when there is no point (a minimum of +inf). */
int oracle_cube_from_bounds(const double bounds[6], double box[4]) {
    if (isinf(bounds[0]) && bounds[0] > 0.0) {
        box[0] = box[1] = box[2] = 0.0;
        box[3] = 1.0;
        return ORACLE_OK;
    }
    double side = 0.0;
    for (int d = 0; d < 3; ++d) {
        box[d] = bounds[d];
        double ext = bounds[3 + d] - bounds[d];
        if (ext > side) side = ext;
    }
    box[3] = (side > 0.0) ? side : 1.0;
    return ORACLE_OK;
}

/* Sec. 6: the domain decomposition groups the leaves into n_ranks bins of consecutive leaves with
 * about N_tot / n_ranks particles each. Reading of "about": the bin of rank r starts at cut r, the
 * first leaf whose preceding leaves hold at least r N_tot / n_ranks particles (compared exactly as
 * integers: prefix * n_ranks >= N_tot * r), n_l when no leaf qualifies; cuts[0] = 0 and
 * cuts[n_ranks] = n_l. Written as the plain scan of the prefix for every cut. */
int oracle_decompose(const uint32_t* N, int64_t nl, int n_ranks, int64_t* cuts) {
    if (nl < 0 || n_ranks < 1) return ORACLE_E_ARG;
    uint64_t total = 0;
    for (int64_t i = 0; i < nl; ++i) total += N[i];
    cuts[0] = 0;
    for (int r = 1; r < n_ranks; ++r) {
        uint64_t prefix = 0;
        int64_t i = 0;
        while (i < nl && !(prefix * (uint64_t)n_ranks >= total * (uint64_t)r)) {
            prefix += N[i];
            ++i;
        }
        cuts[r] = i;
    }
    cuts[n_ranks] = nl;
    return ORACLE_OK;
}

#define GRID_CELLS (1u << L) /* 2^L cells per axis */

/* Scale from coordinates to grid units: 2^L / side, one correctly rounded division. */
double oracle_scale(double side) { return (double)GRID_CELLS / side; }

/* Grid coordinate of one axis (Sec. 3 maps the box onto [0, 2^L)^3): u = (x - lo) * scale with
 * two roundings, then floor, clamped to [0, 2^L - 1]. Points left of the box map to 0, points at
 * or beyond its right face to 2^L - 1. */
uint32_t oracle_grid_coord(double x, double lo, double scale) {
    double u = (x - lo) * scale;
    if (!(u > 0.0)) return 0u;
    if (u >= (double)GRID_CELLS) return GRID_CELLS - 1u;
    return (uint32_t)floor(u);
}

/* Morton (Z-order) key: octal digit i (from the top) holds bit L-i of x, y, z, with x as the
 * most significant bit of the digit. Written as a plain per-level loop. */
uint64_t oracle_morton_key(uint32_t ix, uint32_t iy, uint32_t iz) {
    uint64_t key = 0;
    for (int b = L - 1; b >= 0; --b) {
        uint64_t digit = (uint64_t)(((ix >> b) & 1u) << 2 | ((iy >> b) & 1u) << 1 | ((iz >> b) & 1u));
        key = (key << 3) | digit;
    }
    return key;
}

void oracle_morton_decode(uint64_t key, uint32_t* ix, uint32_t* iy, uint32_t* iz) {
    uint32_t x = 0, y = 0, z = 0;
    for (int b = L - 1; b >= 0; --b) {
        uint32_t digit = (uint32_t)((key >> (3 * b)) & 7u);
        x = (x << 1) | (digit >> 2);
        y = (y << 1) | ((digit >> 1) & 1u);
        z = (z << 1) | (digit & 1u);
    }
    *ix = x;
    *iy = y;
    *iz = z;
}

/* 3D Hilbert key of order `order` (bits per axis). The paper (Sec. 1, Sec. 3) uses "a 3D version
 * of the Hilbert curve" without fixing the variant; this oracle takes J. Skilling's formulation
 * ("Programming the Hilbert curve", AIP Conf. Proc. 707, 2004): the coordinates are brought into
 * the curve's "transposed" form by walking the bit levels from the top, at each level either
 * inverting the lower bits of the first axis or exchanging the lower bits of the first axis and
 * the current one; a Gray code across axes follows. The key interleaves the transposed axes
 * (first axis in the most significant bit of each octal digit). */
uint64_t oracle_hilbert_key_order(uint32_t ix, uint32_t iy, uint32_t iz, int order) {
    uint32_t X[3] = {ix, iy, iz};
    if (order <= 0) return 0;
    uint32_t top = 1u << (order - 1);
    for (uint32_t q = top; q > 1; q >>= 1) {
        uint32_t lower = q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & q) {
                X[0] ^= lower; /* invert the lower bits of the first axis */
            } else {
                uint32_t t = (X[0] ^ X[i]) & lower; /* exchange lower bits of axis 0 and axis i */
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0]; /* Gray code across axes */
    X[2] ^= X[1];
    uint32_t flip = 0;
    for (uint32_t q = top; q > 1; q >>= 1)
        if (X[2] & q) flip ^= q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= flip;

    uint64_t key = 0;
    for (int b = order - 1; b >= 0; --b)
        for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

/* Inverse of oracle_hilbert_key_order: undo the interleave, the Gray code and the per-level
 * inversions/exchanges (walked from the bottom level up). */
void oracle_hilbert_decode_order(uint64_t key, int order, uint32_t* ix, uint32_t* iy, uint32_t* iz) {
    uint32_t X[3] = {0, 0, 0};
    for (int b = order - 1; b >= 0; --b)
        for (int i = 0; i < 3; ++i) X[i] |= (uint32_t)((key >> (3 * b + (2 - i))) & 1u) << b;

    uint32_t t = X[2] >> 1; /* Gray decode */
    X[2] ^= X[1];
    X[1] ^= X[0];
    X[0] ^= t;
    uint32_t end = (order >= 32) ? 0u : (1u << order);
    for (uint32_t q = 2; q != end && q != 0; q <<= 1) {
        uint32_t lower = q - 1;
        for (int i = 2; i >= 0; --i) {
            if (X[i] & q) {
                X[0] ^= lower;
            } else {
                uint32_t s = (X[0] ^ X[i]) & lower;
                X[0] ^= s;
                X[i] ^= s;
            }
        }
    }
    *ix = X[0];
    *iy = X[1];
    *iz = X[2];
}

uint64_t oracle_hilbert_key(uint32_t ix, uint32_t iy, uint32_t iz) {
    return oracle_hilbert_key_order(ix, iy, iz, L);
}

/* Keys of all particles: curve 0 = Morton, 1 = Hilbert. box = {lo_x, lo_y, lo_z, side}. */
int oracle_keys(const double* x, const double* y, const double* z, int64_t n, const double box[4], int curve,
                uint64_t* keys) {
    if (n < 0 || (curve != 0 && curve != 1) || !(box[3] > 0.0)) return ORACLE_E_ARG;
    double scale = oracle_scale(box[3]);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i) {
        if (isnan(x[i]) || isnan(y[i]) || isnan(z[i])) {
            bad = 1;
            continue;
        }
        uint32_t gx = oracle_grid_coord(x[i], box[0], scale);
        uint32_t gy = oracle_grid_coord(y[i], box[1], scale);
        uint32_t gz = oracle_grid_coord(z[i], box[2], scale);
        keys[i] = curve == 0 ? oracle_morton_key(gx, gy, gz) : oracle_hilbert_key(gx, gy, gz);
    }
    return bad ? ORACLE_E_ARG : ORACLE_OK;
}

/* =====================================================================================
 * Sec. 4 and Table 1: sort_by_key of the particle keys with the identity permutation as values.
 * Stable: equal keys keep ascending original index, so sorting the pairs (key, index)
 * lexicographically gives the unique answer.
 * ===================================================================================== */
typedef struct {
    uint64_t key;
    uint32_t idx;
} key_index;

static int cmp_key_index(const void* a, const void* b) {
    const key_index* p = (const key_index*)a;
    const key_index* q = (const key_index*)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
    return 0;
}

int oracle_sort(const uint64_t* keys, int64_t n, uint64_t* sorted, uint32_t* perm) {
    if (n < 0 || n > 0xFFFFFFFFLL) return ORACLE_E_ARG;
    if (n == 0) return ORACLE_OK;
    key_index* a = (key_index*)malloc((size_t)n * sizeof(key_index));
    key_index* tmp = (key_index*)malloc((size_t)n * sizeof(key_index));
    if (!a || !tmp) {
        free(a);
        free(tmp);
        return ORACLE_E_ARG;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        a[i].key = keys[i];
        a[i].idx = (uint32_t)i;
    }
    sort_total(a, tmp, n, sizeof(key_index), cmp_key_index);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        sorted[i] = a[i].key;
        perm[i] = a[i].idx;
    }
    free(a);
    free(tmp);
    return ORACLE_OK;
}

/* =====================================================================================
 * Sec. 4: the cornerstone leaf array.
 * ===================================================================================== */

/* First position in sorted P whose key is >= `key`. */
int64_t oracle_lower_bound(const uint64_t* P, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (P[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

/* Eq. (histogram), f: N_i = number of P in [K_i, K_{i+1}), found as the difference of the two
 * binary-search positions of the bin delimiters. */
int oracle_histogram(const uint64_t* P, int64_t n, const uint64_t* K, int64_t nl, uint32_t* N) {
    if (nl < 1) return ORACLE_E_ARG;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nl; ++i)
        N[i] = (uint32_t)(oracle_lower_bound(P, n, K[i + 1]) - oracle_lower_bound(P, n, K[i]));
    return ORACLE_OK;
}

/* Eq. (g1): rebalance decision O_i for every leaf, O_nl = 0.
 *   O_i = 8 (split) when N_i > Ncrit; a leaf of one key (delta = 1, depth L) cannot be split and
 *         is kept (reading: the paper is silent on full-depth leaves).
 *   O_i = 0 (merge away) when all of
 *         - K_i is not the first octant of its parent: j = (K_i mod 8 delta_i) / delta_i >= 1,
 *         - the 8 siblings are consecutive leaves: K_{i-j} + 8 delta_i = K_{i-j+8},
 *         - their combined count is <= Ncrit (reading: the paper states a strict comparison;
 *           the non-strict one is the reading that agrees with the balance condition of the
 *           converged array, every leaf at most Ncrit and every internal node above it).
 *   O_i = 1 otherwise. */
int oracle_rebalance_decision(const uint64_t* K, const uint32_t* N, int64_t nl, uint32_t ncrit, uint32_t* O) {
    if (nl < 1) return ORACLE_E_ARG;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nl; ++i) {
        uint64_t delta = K[i + 1] - K[i];
        uint32_t op = 1;
        if (N[i] > ncrit && delta > 1) {
            op = 8;
        } else if (delta < KEY_END) {
            uint64_t j = (K[i] % (8 * delta)) / delta;
            if (j >= 1 && (int64_t)j <= i && i - (int64_t)j + 8 <= nl) {
                int64_t first = i - (int64_t)j;
                if (K[first] + 8 * delta == K[first + 8]) {
                    uint64_t sum = 0;
                    for (int64_t s = first; s < first + 8; ++s) sum += N[s];
                    if (sum <= ncrit) op = 0;
                }
            }
        }
        O[i] = op;
    }
    O[nl] = 0;
    return ORACLE_OK;
}

/* Eq. (g2): exclusive prefix sum over len entries; Oprime[len-1] + O[len-1] would be the total. */
int oracle_exclusive_scan(const uint32_t* O, int64_t len, uint64_t* Oprime) {
    uint64_t acc = 0;
    for (int64_t i = 0; i < len; ++i) {
        Oprime[i] = acc;
        acc += O[i];
    }
    return ORACLE_OK;
}

/* Eq. (g3) with Eqs. (rebalancecopy) and (rebalancesplit); the new array ends with 8^L at
 * index O'_nl, the new number of leaves. */
int oracle_rebalance(const uint64_t* K, const uint32_t* O, const uint64_t* Oprime, int64_t nl, uint64_t* Kout) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nl; ++i) {
        uint64_t delta = K[i + 1] - K[i];
        if (O[i] == 1) {
            Kout[Oprime[i]] = K[i];
        } else if (O[i] == 8) {
            for (uint64_t j = 0; j < 8; ++j) Kout[Oprime[i] + j] = K[i] + j * (delta / 8);
        }
    }
    Kout[Oprime[nl]] = KEY_END;
    return ORACLE_OK;
}

/* The f/g iteration of Sec. 4: start from Kinit (or the root {0, 8^L} when nl_init == 0) and
 * apply f then g until g1 reports O_i = 1 for every leaf. iters_out = number of f/g
 * invocations, including the final one that found nothing to change. Nout = final counts. */
int oracle_build_leaves(const uint64_t* P, int64_t n, uint32_t ncrit, const uint64_t* Kinit, int64_t nl_init,
                        uint64_t* Kout, int64_t cap, int64_t* nl_out, uint32_t* Nout, int max_iters,
                        int* iters_out) {
    if (cap < 1 || n < 0) return ORACLE_E_ARG;
    int64_t work_cap = cap * 8 + 8;
    uint64_t* K = (uint64_t*)malloc((size_t)(work_cap + 1) * sizeof(uint64_t));
    uint64_t* Kn = (uint64_t*)malloc((size_t)(work_cap + 1) * sizeof(uint64_t));
    uint32_t* N = (uint32_t*)malloc((size_t)(work_cap + 1) * sizeof(uint32_t));
    uint32_t* O = (uint32_t*)malloc((size_t)(work_cap + 1) * sizeof(uint32_t));
    uint64_t* Op = (uint64_t*)malloc((size_t)(work_cap + 1) * sizeof(uint64_t));
    int rc = ORACLE_OK;
    int64_t nl;
    if (nl_init <= 0) {
        nl = 1;
        K[0] = 0;
        K[1] = KEY_END;
    } else {
        if (nl_init > work_cap) {
            rc = ORACLE_E_CAPACITY;
            goto done;
        }
        nl = nl_init;
        memcpy(K, Kinit, (size_t)(nl + 1) * sizeof(uint64_t));
        if (oracle_check_cornerstone(K, nl) != ORACLE_OK) {
            rc = ORACLE_E_ARG;
            goto done;
        }
    }
    int it = 0;
    for (;;) {
        if (it >= max_iters) {
            rc = ORACLE_E_NOT_CONVERGED;
            break;
        }
        ++it;
        oracle_histogram(P, n, K, nl, N);
        oracle_rebalance_decision(K, N, nl, ncrit, O);
        int changed = 0;
#pragma omp parallel for schedule(static) reduction(| : changed)
        for (int64_t i = 0; i < nl; ++i) changed |= (O[i] != 1);
        if (!changed) break;
        oracle_exclusive_scan(O, nl + 1, Op);
        int64_t nl_new = (int64_t)Op[nl];
        if (nl_new > work_cap) {
            rc = ORACLE_E_CAPACITY;
            *nl_out = nl_new;
            goto done;
        }
        oracle_rebalance(K, O, Op, nl, Kn);
        uint64_t* t = K;
        K = Kn;
        Kn = t;
        nl = nl_new;
    }
    *iters_out = it;
    *nl_out = nl;
    if (rc == ORACLE_OK) {
        if (nl > cap) {
            rc = ORACLE_E_CAPACITY;
        } else {
            memcpy(Kout, K, (size_t)(nl + 1) * sizeof(uint64_t));
            memcpy(Nout, N, (size_t)nl * sizeof(uint32_t));
        }
    }
done:
    free(K);
    free(Kn);
    free(N);
    free(O);
    free(Op);
    return rc;
}

/* Definition of the balanced octree (Sec. 4: leaves hold <= Ncrit particles, internal nodes more
 * than Ncrit), built top-down: a node is split into its 8 octants exactly when it holds more
 * than Ncrit particles and is above the deepest level L. Emits the leaf start keys in SFC order.
 * This is the fixpoint the f/g iteration must reach; the tests compare the two. */
static int canonical_rec(const uint64_t* P, int64_t n, uint32_t ncrit, uint64_t start, int level, uint64_t* Kout,
                         int64_t cap, int64_t* nl) {
    uint64_t size = 1ULL << (3 * (L - level));
    int64_t cnt = oracle_lower_bound(P, n, start + size) - oracle_lower_bound(P, n, start);
    if (cnt > (int64_t)ncrit && level < L) {
        for (uint64_t c = 0; c < 8; ++c) {
            int rc = canonical_rec(P, n, ncrit, start + c * (size / 8), level + 1, Kout, cap, nl);
            if (rc) return rc;
        }
        return ORACLE_OK;
    }
    if (*nl >= cap) return ORACLE_E_CAPACITY;
    Kout[(*nl)++] = start;
    return ORACLE_OK;
}

int oracle_canonical_leaves(const uint64_t* P, int64_t n, uint32_t ncrit, uint64_t* Kout, int64_t cap,
                            int64_t* nl_out) {
    int64_t nl = 0;
    int rc = canonical_rec(P, n, ncrit, 0, 0, Kout, cap, &nl);
    if (rc) return rc;
    Kout[nl] = KEY_END;
    *nl_out = nl;
    return ORACLE_OK;
}

/* Eq. (cstone): K_0 = 0, K_nl = 8^L, strictly increasing, every gap a power of 8 (<= 8^L);
 * additionally each K_i is a multiple of its gap (the key of an octree node, Sec. 3). */
int oracle_check_cornerstone(const uint64_t* K, int64_t nl) {
    if (nl < 1 || K[0] != 0 || K[nl] != KEY_END) return ORACLE_E_INVARIANT;
    for (int64_t i = 0; i < nl; ++i) {
        if (!(K[i] < K[i + 1])) return ORACLE_E_INVARIANT;
        uint64_t d = K[i + 1] - K[i];
        int ok = 0;
        for (int l = 0; l <= L; ++l)
            if (d == (1ULL << (3 * l))) ok = 1;
        if (!ok || K[i] % d != 0) return ORACLE_E_INVARIANT;
    }
    return ORACLE_OK;
}

/* =====================================================================================
 * Sec. 7: locally essential (focused) octree on one process. The focus F is the contiguous key
 * range [f_start, f_end). A node is the key range [s, s + 8^(L-l)) at level l; its cube is the
 * level-l cell holding the first key's grid cell. The minimum-distance MAC of a node holds for
 * every point of F when r_min > l_node / theta, with r_min the smallest distance between the node
 * cube and the cubes that tile F, and l_node the node's edge; both in grid units (cells of the
 * 2^L grid), r_min^2 an exact integer and (l_node / theta)^2 evaluated as two IEEE double roundings.
 * ===================================================================================== */
static void node_cell(uint64_t start, int level, int curve, uint32_t c[3]) {
    uint32_t ix, iy, iz;
    if (curve == 0)
        oracle_morton_decode(start, &ix, &iy, &iz);
    else
        oracle_hilbert_decode_order(start, L, &ix, &iy, &iz);
    int sh = L - level;
    c[0] = (ix >> sh) << sh;
    c[1] = (iy >> sh) << sh;
    c[2] = (iz >> sh) << sh;
}

/* The maximal octree nodes tiling [f_start, f_end), in key order: at each position take the
 * largest node that starts there and ends inside the range. At most 2 * 7 * L nodes. */
int oracle_focus_tiles(uint64_t f_start, uint64_t f_end, uint64_t* tile_start, int* tile_level, int cap) {
    int nt = 0;
    uint64_t s = f_start;
    while (s < f_end) {
        int level = 0;
        for (; level <= L; ++level) {
            uint64_t size = 1ULL << (3 * (L - level));
            if (s % size == 0 && s + size <= f_end) break;
        }
        if (nt >= cap) return ORACLE_E_CAPACITY;
        tile_start[nt] = s;
        tile_level[nt] = level;
        ++nt;
        s += 1ULL << (3 * (L - level));
    }
    return nt;
}

static uint64_t cube_gap2(const uint32_t a[3], uint64_t asz, const uint32_t b[3], uint64_t bsz) {
    uint64_t r2 = 0;
    for (int d = 0; d < 3; ++d) {
        uint64_t a0 = a[d], a1 = a[d] + asz, b0 = b[d], b1 = b[d] + bsz;
        uint64_t gap = 0;
        if (b0 > a1) gap = b0 - a1;
        if (a0 > b1) gap = a0 - b1;
        r2 += gap * gap;
    }
    return r2;
}

int oracle_mac_passes(uint64_t start, int level, uint64_t f_start, uint64_t f_end, double theta, int curve) {
    uint64_t ts[2 * 7 * (L + 1)];
    int tl[2 * 7 * (L + 1)];
    int nt = oracle_focus_tiles(f_start, f_end, ts, tl, 2 * 7 * (L + 1));
    if (nt < 0) return nt;
    uint32_t c[3];
    node_cell(start, level, curve, c);
    uint64_t size = 1ULL << (L - level);
    uint64_t best = UINT64_MAX;
    for (int t = 0; t < nt; ++t) {
        uint32_t tc[3];
        node_cell(ts[t], tl[t], curve, tc);
        uint64_t r2 = cube_gap2(c, size, tc, 1ULL << (L - tl[t]));
        if (r2 < best) best = r2;
    }
    if (nt == 0) return 1; /* an empty focus accepts every node */
    double q = (double)size / theta;
    return (double)best > q * q;
}

/* The node [start, start + size) shares no key with F (always true for an empty F). */
static int outside_focus(uint64_t start, uint64_t size, uint64_t f_start, uint64_t f_end) {
    return f_end <= f_start || start + size <= f_start || start >= f_end;
}

/* g1^LE: inside (or overlapping) F exactly g1; outside F a leaf splits only when it also fails the
 * MAC, and 8 sibling leaves merge when their parent holds at most Ncrit particles or lies outside F
 * and passes the MAC. */
int oracle_focus_decision(const uint64_t* K, const uint32_t* N, int64_t nl, uint32_t ncrit, uint64_t f_start,
                          uint64_t f_end, double theta, int curve, uint32_t* O) {
    if (nl < 1) return ORACLE_E_ARG;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < nl; ++i) {
        uint64_t delta = K[i + 1] - K[i];
        int level = L;
        for (uint64_t d = delta; d > 1; d >>= 3) --level;
        uint32_t op = 1;
        int splittable = N[i] > ncrit && delta > 1;
        if (splittable && outside_focus(K[i], delta, f_start, f_end) &&
            oracle_mac_passes(K[i], level, f_start, f_end, theta, curve))
            splittable = 0;
        if (splittable) {
            op = 8;
        } else if (delta < KEY_END) {
            uint64_t j = (K[i] % (8 * delta)) / delta;
            if (j >= 1 && (int64_t)j <= i && i - (int64_t)j + 8 <= nl) {
                int64_t first = i - (int64_t)j;
                if (K[first] + 8 * delta == K[first + 8]) {
                    uint64_t sum = 0;
                    for (int64_t s2 = first; s2 < first + 8; ++s2) sum += N[s2];
                    int parent_out = outside_focus(K[first], 8 * delta, f_start, f_end);
                    if (sum <= ncrit ||
                        (parent_out && oracle_mac_passes(K[first], level - 1, f_start, f_end, theta, curve)))
                        op = 0;
                }
            }
        }
        O[i] = op;
    }
    O[nl] = 0;
    return ORACLE_OK;
}

/* The literal iteration of f (counts), g1^LE, g2, g3 until nothing changes (Sec. 7, Eqs.
 * histogramf, mac, rebalancef on one process, so f^LE_1 is the plain histogram). */
int oracle_build_focus_leaves(const uint64_t* P, int64_t n, uint32_t ncrit, uint64_t f_start, uint64_t f_end,
                              double theta, int curve, const uint64_t* Kinit, int64_t nl_init, uint64_t* Kout,
                              int64_t cap, int64_t* nl_out, uint32_t* Nout, int max_iters, int* iters_out) {
    if (cap < 1 || n < 0 || !(theta > 0.0)) return ORACLE_E_ARG;
    int64_t work_cap = cap * 8 + 8;
    uint64_t* K = (uint64_t*)malloc((size_t)(work_cap + 1) * sizeof(uint64_t));
    uint64_t* Kn = (uint64_t*)malloc((size_t)(work_cap + 1) * sizeof(uint64_t));
    uint32_t* N = (uint32_t*)malloc((size_t)(work_cap + 1) * sizeof(uint32_t));
    uint32_t* O = (uint32_t*)malloc((size_t)(work_cap + 1) * sizeof(uint32_t));
    uint64_t* Op = (uint64_t*)malloc((size_t)(work_cap + 1) * sizeof(uint64_t));
    int rc = ORACLE_OK;
    int64_t nl;
    if (nl_init <= 0) {
        nl = 1;
        K[0] = 0;
        K[1] = KEY_END;
    } else {
        if (nl_init > work_cap || oracle_check_cornerstone(Kinit, nl_init) != ORACLE_OK) {
            rc = ORACLE_E_ARG;
            goto done;
        }
        nl = nl_init;
        memcpy(K, Kinit, (size_t)(nl + 1) * sizeof(uint64_t));
    }
    int it = 0;
    for (;;) {
        if (it >= max_iters) {
            rc = ORACLE_E_NOT_CONVERGED;
            break;
        }
        ++it;
        oracle_histogram(P, n, K, nl, N);
        oracle_focus_decision(K, N, nl, ncrit, f_start, f_end, theta, curve, O);
        int changed = 0;
#pragma omp parallel for schedule(static) reduction(| : changed)
        for (int64_t i = 0; i < nl; ++i) changed |= (O[i] != 1);
        if (!changed) break;
        oracle_exclusive_scan(O, nl + 1, Op);
        int64_t nl_new = (int64_t)Op[nl];
        if (nl_new > work_cap) {
            rc = ORACLE_E_CAPACITY;
            goto done;
        }
        oracle_rebalance(K, O, Op, nl, Kn);
        uint64_t* t = K;
        K = Kn;
        Kn = t;
        nl = nl_new;
    }
    *iters_out = it;
    *nl_out = nl;
    if (rc == ORACLE_OK) {
        if (nl > cap) {
            rc = ORACLE_E_CAPACITY;
        } else {
            memcpy(Kout, K, (size_t)(nl + 1) * sizeof(uint64_t));
            memcpy(Nout, N, (size_t)nl * sizeof(uint32_t));
        }
    }
done:
    free(K);
    free(Kn);
    free(N);
    free(O);
    free(Op);
    return rc;
}

/* Definition of the focused tree, top-down: a node is split exactly when it is above level L,
 * holds more than Ncrit particles, and overlaps F or fails the MAC. */
static int canonical_focus_rec(const uint64_t* P, int64_t n, uint32_t ncrit, uint64_t f_start, uint64_t f_end,
                               double theta, int curve, uint64_t start, int level, uint64_t* Kout, int64_t cap,
                               int64_t* nl) {
    uint64_t size = 1ULL << (3 * (L - level));
    int64_t cnt = oracle_lower_bound(P, n, start + size) - oracle_lower_bound(P, n, start);
    int split = cnt > (int64_t)ncrit && level < L;
    if (split && outside_focus(start, size, f_start, f_end) &&
        oracle_mac_passes(start, level, f_start, f_end, theta, curve))
        split = 0;
    if (split) {
        for (uint64_t c = 0; c < 8; ++c) {
            int rc = canonical_focus_rec(P, n, ncrit, f_start, f_end, theta, curve, start + c * (size / 8), level + 1,
                                         Kout, cap, nl);
            if (rc) return rc;
        }
        return ORACLE_OK;
    }
    if (*nl >= cap) return ORACLE_E_CAPACITY;
    Kout[(*nl)++] = start;
    return ORACLE_OK;
}

int oracle_canonical_focus_leaves(const uint64_t* P, int64_t n, uint32_t ncrit, uint64_t f_start, uint64_t f_end,
                                  double theta, int curve, uint64_t* Kout, int64_t cap, int64_t* nl_out) {
    int64_t nl = 0;
    int rc = canonical_focus_rec(P, n, ncrit, f_start, f_end, theta, curve, 0, 0, Kout, cap, &nl);
    if (rc) return rc;
    Kout[nl] = KEY_END;
    *nl_out = nl;
    return ORACLE_OK;
}

/* =====================================================================================
 * Sec. 5: fully linked octree in breadth-first order.
 * Node keys use the Warren-Salmon placeholder-bit format: a 1 bit followed by the node's
 * `level` octal digits. The node set of the tree defined by K is every leaf plus every proper
 * ancestor of a leaf. Sorting the placeholder keys ascending orders them by level first and by
 * SFC position within a level: the breadth-first layout of Sec. 5, step 3.
 * ===================================================================================== */
static int leaf_level(uint64_t delta) {
    int l = L;
    while (delta > 1) {
        delta >>= 3;
        --l;
    }
    return l;
}

static uint64_t placeholder(uint64_t key, int level) {
    return (1ULL << (3 * level)) | (key >> (3 * (L - level)));
}

static int placeholder_level(uint64_t nk) {
    int msb = 63;
    while (!((nk >> msb) & 1ULL)) --msb;
    return msb / 3;
}

static int cmp_u64(const void* a, const void* b) {
    uint64_t p = *(const uint64_t*)a, q = *(const uint64_t*)b;
    return (p > q) - (p < q);
}

/* Ascending order of n 64-bit words (equal words end up adjacent; the caller removes repeats). */
static void sort_total_u64(uint64_t* a, uint64_t* tmp, int64_t n) { sort_total(a, tmp, n, sizeof(uint64_t), cmp_u64); }

static int64_t find_u64(const uint64_t* a, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < n && a[lo] == v) ? lo : -1;
}

/* Outputs, n = nl + (nl - 1) / 7 nodes:
 *   NK[n]           placeholder keys, breadth-first
 *   CO[n]           index of the first of the 8 children, 0 for a leaf
 *   LO[L + 2]       LO[l] = index of the first node of level l, LO[L+1] = n
 *   leaf_to_node[nl] node index of leaf i
 *   parent[(n-1)/8] parent index of the sibling group g = nodes 1+8g .. 8+8g (may be NULL) */
int oracle_link(const uint64_t* K, int64_t nl, uint64_t* NK, int32_t* CO, int32_t* LO, int32_t* leaf_to_node,
                int32_t* parent) {
    if (nl < 1 || (nl - 1) % 7 != 0) return ORACLE_E_ARG;
    int64_t n_expected = nl + (nl - 1) / 7;
    int64_t cap = nl * (L + 1);
    uint64_t* all = (uint64_t*)malloc((size_t)cap * sizeof(uint64_t));
    int64_t cnt = 0;
    for (int64_t i = 0; i < nl; ++i) {
        int lev = leaf_level(K[i + 1] - K[i]);
        for (int a = 0; a <= lev; ++a) all[cnt++] = placeholder(K[i], a);
    }
    uint64_t* tmp = (uint64_t*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(uint64_t));
    sort_total_u64(all, tmp, cnt);
    free(tmp);
    int64_t n = 0;
    for (int64_t i = 0; i < cnt; ++i)
        if (n == 0 || all[i] != all[n - 1]) all[n++] = all[i];
    if (n != n_expected) {
        free(all);
        return ORACLE_E_INVARIANT;
    }
    memcpy(NK, all, (size_t)n * sizeof(uint64_t));
    free(all);

    for (int l = 0; l <= L; ++l) {
        uint64_t first = 1ULL << (3 * l);
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (NK[mid] < first)
                lo = mid + 1;
            else
                hi = mid;
        }
        LO[l] = (int32_t)lo;
    }
    LO[L + 1] = (int32_t)n;

    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i) {
        int lev = placeholder_level(NK[i]);
        int64_t c = (lev < L) ? find_u64(NK, n, NK[i] << 3) : -1;
        CO[i] = (c < 0) ? 0 : (int32_t)c;
        if (c >= 0) {
            if ((c - 1) % 8 != 0) {
                bad = 1;
                continue;
            }
            for (int j = 0; j < 8; ++j)
                if (c + j >= n || NK[c + j] != ((NK[i] << 3) | (uint64_t)j)) bad = 1;
            if (parent) parent[(c - 1) / 8] = (int32_t)i;
        }
    }
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < nl; ++i) {
        int lev = leaf_level(K[i + 1] - K[i]);
        int64_t v = find_u64(NK, n, placeholder(K[i], lev));
        if (v < 0) {
            bad = 1;
            continue;
        }
        leaf_to_node[i] = (int32_t)v;
    }
    return bad ? ORACLE_E_INVARIANT : ORACLE_OK;
}

/* Key range [start, end) covered by a placeholder node key. */
static void node_range(uint64_t nk, uint64_t* start, uint64_t* end) {
    int lev = placeholder_level(nk);
    uint64_t prefix = nk ^ (1ULL << (3 * lev));
    *start = prefix << (3 * (L - lev));
    *end = *start + (1ULL << (3 * (L - lev)));
}

/* Node particle counts (Sec. 5, node properties): the number of sorted keys inside each node's
 * key range, by definition. */
int oracle_node_counts(const uint64_t* P, int64_t n, const uint64_t* NK, int64_t nnodes, uint32_t* counts) {
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < nnodes; ++v) {
        uint64_t s, e;
        node_range(NK[v], &s, &e);
        counts[v] = (uint32_t)(oracle_lower_bound(P, n, e) - oracle_lower_bound(P, n, s));
    }
    return ORACLE_OK;
}

/* Monopole and quadrupole of selected nodes (Sec. 5 node properties; Sec. 8 uses Cartesian
 * expansions up to the quadrupole), in double precision, directly over each node's particles:
 *   M      = sum m_p
 *   com    = sum m_p x_p / M                                   (expansion centre)
 *   quad   = sum m_p (x_p - com)_a (x_p - com)_b, components xx, xy, xz, yy, yz, zz
 * An empty node has M = 0, com = 0, quad = 0 (reading: the paper does not define it).
 * Particles of a node are the sorted positions [lb(start), lb(end)); perm maps them back to the
 * input arrays. nodes[k] selects the node whose results go to row k. */
int oracle_multipoles(const double* x, const double* y, const double* z, const float* m, const uint64_t* P,
                      const uint32_t* perm, int64_t n, const uint64_t* NK, const int64_t* nodes, int64_t nsel,
                      double* M, double* com, double* quad) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t k = 0; k < nsel; ++k) {
        uint64_t s, e;
        node_range(NK[nodes[k]], &s, &e);
        int64_t a = oracle_lower_bound(P, n, s), b = oracle_lower_bound(P, n, e);
        double mass = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
        for (int64_t j = a; j < b; ++j) {
            uint32_t p = perm[j];
            double mp = (double)m[p];
            mass += mp;
            cx += mp * x[p];
            cy += mp * y[p];
            cz += mp * z[p];
        }
        double q[6] = {0, 0, 0, 0, 0, 0};
        if (b > a && mass > 0.0) {
            cx /= mass;
            cy /= mass;
            cz /= mass;
            for (int64_t j = a; j < b; ++j) {
                uint32_t p = perm[j];
                double mp = (double)m[p];
                double dx = x[p] - cx, dy = y[p] - cy, dz = z[p] - cz;
                q[0] += mp * dx * dx;
                q[1] += mp * dx * dy;
                q[2] += mp * dx * dz;
                q[3] += mp * dy * dy;
                q[4] += mp * dy * dz;
                q[5] += mp * dz * dz;
            }
        } else {
            cx = cy = cz = 0.0;
        }
        M[k] = mass;
        com[3 * k + 0] = cx;
        com[3 * k + 1] = cy;
        com[3 * k + 2] = cz;
        for (int c = 0; c < 6; ++c) quad[6 * k + c] = q[c];
    }
    return ORACLE_OK;
}
