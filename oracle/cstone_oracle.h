/*
 * Plain CPU oracle for the Cornerstone octree build (Keller et al., PASC'23).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links or calls this code;
 * only the test-suite, the smoke check and the CPU-baseline leg of the benchmark use it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Every routine is the plain definition (or the paper's algorithm step by step), in double
 * precision where floating point is involved, compiled without FMA contraction
 * (-ffp-contract=off) so that every floating-point operation is one IEEE round-to-nearest
 * operation. Loops over independent particles, leaves or nodes may run on several threads
 * (OpenMP); each iteration does the same operations in the same order, so the results are those
 * of the sequential program.
 *
 * Notation follows the paper: L octree levels (L = 21: 63-bit keys; the same source compiled
 * with -DORACLE_L=10 gives the 30-bit keys of Sec. 3's other choice), K = cornerstone array,
 * P = sorted particle keys, N = leaf counts, O / O' = rebalance ops and their exclusive
 * scan, NK / CO / LO = node keys, first-child indices and level offsets.
 *
 * Return convention: 0 = success, negative = error (see ORACLE_E_*).
 */
#ifndef CSTONE_ORACLE_H
#define CSTONE_ORACLE_H

#include <stdint.h>

#ifndef ORACLE_L
#define ORACLE_L 21
#endif

#define ORACLE_OK 0
#define ORACLE_E_ARG (-1)
#define ORACLE_E_CAPACITY (-2)
#define ORACLE_E_NOT_CONVERGED (-3)
#define ORACLE_E_INVARIANT (-4)

/* Threads of the oracle's parallel loops (<= 0: all cores; 1: the sequential program). Results do
 * not depend on it. */
void oracle_set_threads(int threads);
int oracle_get_threads(void);

/* ---- Sec. 3: grid coordinates and space-filling-curve keys ---- */
int oracle_bounding_cube(const double* x, const double* y, const double* z, int64_t n, double box[4]);
uint32_t oracle_grid_coord(double x, double lo, double scale);
double oracle_scale(double side);
uint64_t oracle_morton_key(uint32_t ix, uint32_t iy, uint32_t iz);
void oracle_morton_decode(uint64_t key, uint32_t* ix, uint32_t* iy, uint32_t* iz);
uint64_t oracle_hilbert_key_order(uint32_t ix, uint32_t iy, uint32_t iz, int order);
void oracle_hilbert_decode_order(uint64_t key, int order, uint32_t* ix, uint32_t* iy, uint32_t* iz);
uint64_t oracle_hilbert_key(uint32_t ix, uint32_t iy, uint32_t iz);
int oracle_keys(const double* x, const double* y, const double* z, int64_t n, const double box[4], int curve,
                uint64_t* keys);

/* ---- Sec. 4 / Table 1: stable sort_by_key with the identity permutation ---- */
int oracle_sort(const uint64_t* keys, int64_t n, uint64_t* sorted, uint32_t* perm);

/* ---- Sec. 4: cornerstone leaf array ---- */
int64_t oracle_lower_bound(const uint64_t* P, int64_t n, uint64_t key);
int oracle_histogram(const uint64_t* P, int64_t n, const uint64_t* K, int64_t nl, uint32_t* N);
int oracle_rebalance_decision(const uint64_t* K, const uint32_t* N, int64_t nl, uint32_t ncrit, uint32_t* O);
int oracle_exclusive_scan(const uint32_t* O, int64_t len, uint64_t* Oprime);
int oracle_rebalance(const uint64_t* K, const uint32_t* O, const uint64_t* Oprime, int64_t nl, uint64_t* Kout);
int oracle_build_leaves(const uint64_t* P, int64_t n, uint32_t ncrit, const uint64_t* Kinit, int64_t nl_init,
                        uint64_t* Kout, int64_t cap, int64_t* nl_out, uint32_t* Nout, int max_iters,
                        int* iters_out);
int oracle_canonical_leaves(const uint64_t* P, int64_t n, uint32_t ncrit, uint64_t* Kout, int64_t cap,
                            int64_t* nl_out);
int oracle_check_cornerstone(const uint64_t* K, int64_t nl);

/* ---- Sec. 7: locally essential octree focused on the key range [f_start, f_end) ---- */
int oracle_focus_tiles(uint64_t f_start, uint64_t f_end, uint64_t* tile_start, int* tile_level, int cap);
int oracle_mac_passes(uint64_t start, int level, uint64_t f_start, uint64_t f_end, double theta, int curve);
int oracle_focus_decision(const uint64_t* K, const uint32_t* N, int64_t nl, uint32_t ncrit, uint64_t f_start,
                          uint64_t f_end, double theta, int curve, uint32_t* O);
int oracle_build_focus_leaves(const uint64_t* P, int64_t n, uint32_t ncrit, uint64_t f_start, uint64_t f_end,
                              double theta, int curve, const uint64_t* Kinit, int64_t nl_init, uint64_t* Kout,
                              int64_t cap, int64_t* nl_out, uint32_t* Nout, int max_iters, int* iters_out);
int oracle_canonical_focus_leaves(const uint64_t* P, int64_t n, uint32_t ncrit, uint64_t f_start, uint64_t f_end,
                                  double theta, int curve, uint64_t* Kout, int64_t cap, int64_t* nl_out);

/* ---- Sec. 6: distributed octree and domain decomposition ---- */
int oracle_cube_from_bounds(const double bounds[6], double box[4]);
int oracle_decompose(const uint32_t* N, int64_t nl, int n_ranks, int64_t* cuts);

/* ---- Sec. 5: fully linked octree ---- */
int oracle_link(const uint64_t* K, int64_t nl, uint64_t* NK, int32_t* CO, int32_t* LO, int32_t* leaf_to_node,
                int32_t* parent);

/* ---- Sec. 5 / Sec. 7: node properties ---- */
int oracle_node_counts(const uint64_t* P, int64_t n, const uint64_t* NK, int64_t nnodes, uint32_t* counts);
int oracle_multipoles(const double* x, const double* y, const double* z, const float* m, const uint64_t* P,
                      const uint32_t* perm, int64_t n, const uint64_t* NK, const int64_t* nodes, int64_t nsel,
                      double* M, double* com, double* quad);

#endif
