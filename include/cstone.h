/*
 * cstone.h - C ABI of the GB300-native Cornerstone octree build.
 *
 * Method: S. Keller et al., "Cornerstone: Octree Construction Algorithms for Scalable Particle
 * Simulations", PASC'23 (arXiv 2307.06345). Section references below are to that paper.
 *
 * Conventions shared by every entry point:
 *  - Pointers to arrays are DEVICE pointers (cudaMalloc / torch CUDA memory) owned by the caller,
 *    unless the comment says "host". The library never allocates device memory: scratch space
 *    comes from a caller-provided workspace `ws` of at least the size reported by the matching
 *    *_workspace_size query, 256-byte aligned. A workspace may be reused by later calls on the
 *    same stream but must not be shared by calls that can run concurrently.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Calls are
 *    asynchronous on that stream unless a host out-parameter forces a synchronisation (stated).
 *  - Every function returns a cstone_status. No C++ exception crosses the ABI. On failure a
 *    human-readable detail is available from cstone_last_error_detail (per host thread).
 *  - Keys are 63-bit space-filling-curve keys (L = 21 levels, Sec. 3) stored in uint64_t; the
 *    end of the key space 8^L = 2^63 terminates cornerstone arrays (Eq. cstone).
 *  - Particle counts n must satisfy 0 <= n < 2^30.
 */
#ifndef CSTONE_H
#define CSTONE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CSTONE_API __attribute__((visibility("default")))
#else
#define CSTONE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define CSTONE_LEVELS 21   /* L of the 63-bit keys (entry points cstone_*) */
#define CSTONE30_LEVELS 10 /* L of the 30-bit keys (entry points cstone30_*) */
#define CSTONE_MAX_PARTICLES ((int64_t)1 << 30)
#define CSTONE_MAX_LEAVES ((int64_t)1 << 28)

typedef enum {
    CSTONE_OK = 0,
    CSTONE_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, misaligned or too small workspace */
    CSTONE_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
    CSTONE_ERR_CAPACITY = 3,      /* an output array is too small; the required size is reported */
    CSTONE_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up (results are invalid) */
    CSTONE_ERR_NOT_CONVERGED = 5  /* the rebalance loop hit max_iters */
} cstone_status;

typedef enum { CSTONE_MORTON = 0, CSTONE_HILBERT = 1 } cstone_curve;

/* Static description of a status code. Never NULL. */
CSTONE_API const char* cstone_status_string(int status);

/* Copies the detail message of the last failure on this host thread into buf (NUL-terminated,
 * truncated to len). Returns CSTONE_OK. */
CSTONE_API int cstone_last_error_detail(char* buf, size_t len);

/* Library version as major * 10000 + minor * 100 + patch. */
CSTONE_API int cstone_version(void);

/* Number of kernels this library has launched in this process so far, over all threads and
 * devices (instrumentation; the paper has no counterpart). A launch that failed to start is
 * counted too. */
CSTONE_API int64_t cstone_kernel_launches(void);

/* Reads the device error word kept in the header of any workspace filled by an asynchronous call
 * (cstone_sort, cstone_link_tree) and stores the corresponding status in *status (host).
 * Synchronises `stream`. The word is cleared by the next call that uses the workspace. */
CSTONE_API int cstone_workspace_status(const void* ws, void* stream, int* status);

/* ------------------------------------------------------------------------------------------
 * Bounding cube (the paper is silent on the normalisation of coordinates to the key grid of
 * Sec. 3; this library uses the cube anchored at the per-axis minimum whose side is the largest
 * per-axis extent, side 1 when that extent is 0 or n == 0).
 *   x, y, z  [n] float64 particle coordinates (finite).
 *   box      [4] float64 output: {lo_x, lo_y, lo_z, side}.
 * ------------------------------------------------------------------------------------------ */
CSTONE_API int cstone_bbox_workspace_size(int64_t n, size_t* bytes);
CSTONE_API int cstone_bbox(const double* x, const double* y, const double* z, int64_t n, double* box, void* ws, size_t ws_bytes,
                void* stream);

/* Per-axis bounds of the points: bounds[6] (device) = {min x, min y, min z, max x, max y, max z};
 * with n = 0 the minima are +inf and the maxima -inf. A set spread over several processes takes
 * the minimum and maximum of these over the processes and forms the same bounding cube as
 * cstone_bbox (lo = minima, side = largest extent, 1 if zero). Workspace as for cstone_bbox.
 * Asynchronous. */
CSTONE_API int cstone_bounds(const double* x, const double* y, const double* z, int64_t n, double* bounds, void* ws,
                             size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------------------
 * SFC keys (Sec. 3). Each coordinate is mapped to a grid cell of [0, 2^21) per axis by
 * g = clamp(floor((x - lo) * s), 0, 2^21 - 1) with s = 2^21 / side, the subtraction and the
 * product each rounded once in IEEE double precision (so results match any IEEE host bit for
 * bit); points outside the box are clamped to its faces. The cell is then encoded as a Morton key
 * (octal digit i holds bit 21-i of x, y, z, x most significant) or as a 3D Hilbert key
 * (J. Skilling's formulation of the Hilbert curve, whose level-i prefix is the level-i octree
 * node, Sec. 3).
 *   box   [4] float64 device array {lo_x, lo_y, lo_z, side}, side > 0.
 *   keys  [n] uint64 output.
 * NaN coordinates give unspecified keys.
 * ------------------------------------------------------------------------------------------ */
CSTONE_API int cstone_keys(const double* x, const double* y, const double* z, int64_t n, const double* box, int curve,
                uint64_t* keys, void* stream);

/* ------------------------------------------------------------------------------------------
 * Radix sort_by_key of the particle keys with the identity permutation as values (Sec. 4;
 * Table 1 caption). Stable: equal keys keep ascending input index. LSD, 8-bit digits; every pass
 * counts the digits of every tile, scans the counts and scatters each tile's digit runs.
 *   keys_in   [n] uint64 input keys (may alias keys_out).
 *   keys_out  [n] uint64 sorted keys P.
 *   perm      [n] uint32 output: keys_out[j] = keys_in[perm[j]].
 * Asynchronous; no device wait is involved.
 * ------------------------------------------------------------------------------------------ */
CSTONE_API int cstone_sort_workspace_size(int64_t n, size_t* bytes);
CSTONE_API int cstone_sort(const uint64_t* keys_in, uint64_t* keys_out, uint32_t* perm, int64_t n, void* ws, size_t ws_bytes,
                void* stream);

/* ------------------------------------------------------------------------------------------
 * Sort that allocates nothing (the paper has no counterpart; this is a deployment variant of
 * cstone_sort with the same result). It is for callers that cannot call cudaMalloc and cannot
 * hand out a workspace: code that runs inside a memory allocator's own callbacks, or inside a
 * framework that owns and budgets all device memory of the process, where a new allocation is
 * not allowed. Its scratch is a fixed static device array inside this library (about 13 MB,
 * held on every GPU that loads the library until the process exits), so n is limited to
 * CSTONE_SORT_STATIC_MAX_KEYS; a larger n returns CSTONE_ERR_INVALID_ARG without touching the
 * GPU. The first call on a device looks up the array's device address (cudaGetSymbolAddress):
 * make that first call before any stream capture. All calls share the one array, so calls that
 * can overlap on the GPU (other streams, other host threads) race and must be serialised by the
 * caller. Each call clears what has to start at zero; otherwise the array keeps the last call's
 * intermediate keys, permutation and digit counts, which the next call overwrites before reading.
 * The device address is cached per device ordinal for the life of the process: it does not
 * survive cudaDeviceReset (or any teardown of the primary context) in the host application.
 * `stream` must belong to the current device; a stream of another device returns
 * CSTONE_ERR_INVALID_ARG.
 *   keys_in, keys_out, perm, n, stream: as for cstone_sort (keys_in may alias keys_out).
 * Asynchronous.
 * ------------------------------------------------------------------------------------------ */
#define CSTONE_SORT_STATIC_MAX_KEYS ((int64_t)1 << 20)
CSTONE_API int cstone_sort_static(const uint64_t* keys_in, uint64_t* keys_out, uint32_t* perm, int64_t n,
                                  void* stream);

/* ------------------------------------------------------------------------------------------
 * Cornerstone leaf array (Sec. 4, Eqs. cstone, histogram, g1-g3): starting from the root
 * {0, 8^L} (when *n_leaves == 0 on entry) or from the caller's array in `leaves` (when
 * *n_leaves > 0: warm start from a previous step's leaves, Sec. 4), apply the histogram f and
 * the rebalance g = g3 . g2 . g1 until g1 decides O_i = 1 for every leaf. Rules of g1: split when
 * N_i > ncrit (unless the leaf is a single key at depth L); merge the 8 consecutive sibling
 * leaves of a parent when their combined count is <= ncrit (the first octant keeps its key).
 *   sorted_keys [n] uint64 sorted particle keys P (< 2^63).
 *   leaves      [leaf_cap + 1] uint64 in/out cornerstone array K.
 *   n_leaves    host in/out: leaves on entry (0 = root), final n_l on exit; on
 *               CSTONE_ERR_CAPACITY the number of leaves that did not fit.
 *   counts      [leaf_cap] uint32 output N_i of the final leaves.
 *   offsets     [leaf_cap + 1] uint32 output (may be NULL): offsets[i] = first sorted particle of
 *               leaf i, offsets[n_l] = n.
 *   max_iters   bound on f/g passes (<= 256); iters (host, may be NULL) receives the number of
 *               passes, including the last one that changed nothing.
 * Synchronises `stream` (the host outputs need the converged size).
 * ------------------------------------------------------------------------------------------ */
CSTONE_API int cstone_leaves_workspace_size(int64_t n, int64_t leaf_cap, int32_t max_iters, size_t* bytes);
CSTONE_API int cstone_build_leaves(const uint64_t* sorted_keys, int64_t n, uint32_t ncrit, uint64_t* leaves, int64_t leaf_cap,
                        int64_t* n_leaves, uint32_t* counts, uint32_t* offsets, int32_t max_iters, int32_t* iters,
                        void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------------------
 * Fully linked octree (Sec. 5): all nodes of the tree whose leaves are K, n = n_l + (n_l-1)/7
 * of them, in breadth-first order (by level, then by key), each internal node with exactly 8
 * children.
 *   leaves        [n_leaves + 1] uint64 cornerstone array K.
 *   node_keys     [n] uint64 NK: Warren-Salmon placeholder keys, (1 << 3*level) | key prefix.
 *   child         [n] int32 CO: index of the first of the 8 children, 0 for a leaf.
 *   level_offsets [23] int32 LO: first node of level l = 0..21; LO[22] = n.
 *   leaf_to_node  [n_leaves] int32: node index of leaf i.
 *   parent        [(n-1)/8] int32 (may be NULL): parent of the sibling group g, i.e. of the
 *                 nodes 1+8g .. 8+8g.
 * Asynchronous.
 * ------------------------------------------------------------------------------------------ */
CSTONE_API int cstone_link_workspace_size(int64_t n_leaves, size_t* bytes);
CSTONE_API int cstone_link_tree(const uint64_t* leaves, int64_t n_leaves, uint64_t* node_keys, int32_t* child,
                     int32_t* level_offsets, int32_t* leaf_to_node, int32_t* parent, void* ws, size_t ws_bytes,
                     void* stream);

/* ------------------------------------------------------------------------------------------
 * Node-count upsweep (Sec. 5 node properties, computed by an upward pass as in Sec. 7): a leaf
 * holds its N_i, an internal node the sum of its 8 children. Inputs are the outputs of
 * cstone_build_leaves (counts) and cstone_link_tree (leaf_to_node, child, level_offsets).
 *   node_counts [n] uint32 output.
 * One cooperative launch walking the levels from the deepest; asynchronous. The workspace holds
 * the grid barrier and a list of the internal nodes (4 bytes each). A child array off the linked
 * layout (child[x] = 8 g + 1 for the g-th internal node) is reported in the error word.
 * ------------------------------------------------------------------------------------------ */
CSTONE_API int cstone_upsweep_workspace_size(int64_t n_leaves, size_t* bytes);
CSTONE_API int cstone_upsweep_counts(const uint32_t* leaf_counts, int64_t n_leaves, const int32_t* leaf_to_node,
                                     const int32_t* child, const int32_t* level_offsets, uint32_t* node_counts,
                                     void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------------------
 * Multipole upsweep (Sec. 5 node properties; Sec. 8 uses Cartesian expansions up to the
 * quadrupole): per node the mass M, the centre of mass (expansion centre) and the second
 * moments about it Q_ab = sum m (x - com)_a (x - com)_b, components xx, xy, xz, yy, yz, zz.
 * Accumulation is in FP32 with two-sum compensation (a sum/compensation pair per moment, carried
 * up the tree); positions are taken into 64-bit fixed point so that coordinate differences are
 * exact before their conversion to FP32 (correctly rounded below 2^31 fixed-point units, within one
 * unit in the last place above), and the centre is written in FP64. An empty node has M = 0,
 * com = 0, Q = 0. The workspace holds a 32-byte record per particle, the per-node sums and the list
 * of internal nodes.
 *   x, y, z, m   [n] float64 coordinates and float32 masses in input order.
 *   perm         [n] uint32 sort permutation (cstone_sort).
 *   offsets      [n_leaves + 1] uint32 leaf particle offsets (cstone_build_leaves).
 *   leaf_to_node, child, level_offsets  from cstone_link_tree.
 *   box          [4] float64 device array {lo_x, lo_y, lo_z, side}; it fixes the 64-bit
 *                fixed-point frame of the positions. Every |coordinate| must stay below 2^E, the
 *                smallest power of two above max(|lo|, |lo + 2 side|) (true for any point within
 *                the box); otherwise the workspace error word reports CSTONE_ERR_INVALID_ARG.
 *   mass         [nn] float32, com [3 * nn] float64 (SoA: x block, y block, z block),
 *   quad         [6 * nn] float32 (SoA, component-major), nn = number of nodes.
 * Asynchronous.
 * ------------------------------------------------------------------------------------------ */
CSTONE_API int cstone_multipole_workspace_size(int64_t n, int64_t n_leaves, size_t* bytes);
CSTONE_API int cstone_upsweep_multipoles(const double* x, const double* y, const double* z, const float* m,
                                         const uint32_t* perm, int64_t n, const uint32_t* offsets, int64_t n_leaves,
                                         const int32_t* leaf_to_node, const int32_t* child,
                                         const int32_t* level_offsets, const double* box, float* mass, double* com,
                                         float* quad, void* ws, size_t ws_bytes, void* stream);

/* Keys and multipole records in one read of the coordinates. The paper has no counterpart: it is
 * the keys step (Sec. 3) fused with the first step of the multipole upsweep above, so that x, y, z
 * are read once for both. keys are those of cstone_keys for the same box and curve; records
 * receives one 32-byte record per particle (64-bit fixed-point position in the frame fixed by box,
 * and the mass; the layout is private to the library), which cstone_upsweep_multipoles_records
 * reads in place of x, y, z, m.
 *   m        [n] float32 masses (4-byte aligned).
 *   records  cstone_records_size(n) bytes of device memory, 16-byte aligned, owned by the caller.
 *   ws       cstone_keys_records_workspace_size bytes (256-byte aligned); its error word reports
 *            CSTONE_ERR_INVALID_ARG for a coordinate outside the fixed-point range of box (the
 *            condition of cstone_upsweep_multipoles); read it with cstone_workspace_status.
 * Asynchronous. */
CSTONE_API int cstone_records_size(int64_t n, size_t* bytes);
CSTONE_API int cstone_keys_records_workspace_size(size_t* bytes);
CSTONE_API int cstone_keys_records(const double* x, const double* y, const double* z, const float* m, int64_t n,
                                   const double* box, int curve, uint64_t* keys, void* records, void* ws,
                                   size_t ws_bytes, void* stream);

/* The multipole upsweep from records written by cstone_keys_records with the same box (the pack
 * step skipped); results are bit for bit those of cstone_upsweep_multipoles on the same particles.
 * ws: cstone_multipole_workspace_size(0, n_leaves, &bytes) bytes (no record area). Other arguments
 * as for cstone_upsweep_multipoles. Asynchronous. */
CSTONE_API int cstone_upsweep_multipoles_records(const void* records, const uint32_t* perm, int64_t n,
                                                 const uint32_t* offsets, int64_t n_leaves,
                                                 const int32_t* leaf_to_node, const int32_t* child,
                                                 const int32_t* level_offsets, const double* box, float* mass,
                                                 double* com, float* quad, void* ws, size_t ws_bytes, void* stream);

/* ==========================================================================================
 * Batched builds: S independent particle sets stored back to back (set s owns particles
 * [set_offsets[s], set_offsets[s+1])), built with one launch per phase for all sets. The
 * per-set results equal those of the single-set entry points on each set alone. Offsets arrays
 * named *_offsets are DEVICE int64 arrays of S+1 entries.
 * ========================================================================================== */

/* Bounding cube of every set: boxes [S][4] float64 (device) output. Asynchronous. */
CSTONE_API int cstone_bbox_batched(const double* x, const double* y, const double* z, const int64_t* set_offsets,
                                   int32_t n_sets, double* boxes, void* stream);

/* Keys of all particles, each with its own set's box (boxes [S][4], device). Asynchronous. */
CSTONE_API int cstone_keys_batched_workspace_size(int32_t n_sets, size_t* bytes);
CSTONE_API int cstone_keys_batched(const double* x, const double* y, const double* z, int64_t n,
                                   const int64_t* set_offsets, int32_t n_sets, const double* boxes, int curve,
                                   uint64_t* keys, void* ws, size_t ws_bytes, void* stream);

/* Stable sort of every segment's keys (segments given by seg_offsets), one set of launches per
 * digit pass for all segments: tiles are aligned to segments and digits are offset per segment.
 * perm holds global input indices. keys_in must not alias keys_out. Asynchronous. */
CSTONE_API int cstone_sort_segmented_workspace_size(int64_t n, int32_t n_segs, size_t* bytes);
CSTONE_API int cstone_sort_segmented(const uint64_t* keys_in, uint64_t* keys_out, uint32_t* perm, int64_t n,
                                     const int64_t* seg_offsets, int32_t n_segs, void* ws, size_t ws_bytes,
                                     void* stream);

/* Cornerstone arrays of all sets (Sec. 4) in one cooperative launch. The arrays are stored back to
 * back as "elements": set s owns elements [element_offsets[s], element_offsets[s+1]), its leaves
 * followed by its end key 8^L, so set s has element_offsets[s+1] - element_offsets[s] - 1 leaves.
 *   sorted_keys   [n] keys sorted within each set (cstone_sort_segmented).
 *   elements      [elem_cap] uint64 in/out: on entry the previous arrays when *n_elements > 0
 *                 (warm start, with element_offsets filled in), else ignored (every set starts
 *                 from its root).
 *   element_offsets [S+1] int64 device in/out.
 *   n_elements    host in/out: elements on entry (0 = cold), on exit; on CSTONE_ERR_CAPACITY the
 *                 number of elements that did not fit.
 *   counts        [elem_cap] uint32: leaf counts (0 at end keys); offsets [elem_cap] uint32 (may be
 *                 NULL): first sorted particle (global index) of each element.
 * Synchronises `stream`. */
CSTONE_API int cstone_leaves_batched_workspace_size(int64_t elem_cap, int32_t max_iters, size_t* bytes);
CSTONE_API int cstone_build_leaves_batched(const uint64_t* sorted_keys, int64_t n, const int64_t* set_offsets,
                                           int32_t n_sets, uint32_t ncrit, uint64_t* elements, int64_t elem_cap,
                                           int64_t* element_offsets, int64_t* n_elements, uint32_t* counts,
                                           uint32_t* offsets, int32_t max_iters, int32_t* iters, void* ws,
                                           size_t ws_bytes, void* stream);

/* The batched leaf loop without any host synchronisation, so that it can be captured in a CUDA
 * graph together with the phases before and after it (the time-step driver replays one graph per
 * step). Arguments as for cstone_build_leaves_batched, except:
 *   warm      0: every set starts from its root; else the previous arrays are in `elements` and
 *             `element_offsets`, and their element count is element_offsets[n_sets] (read on the
 *             device).
 * Nothing is returned to the host: the element count of the result is element_offsets[n_sets]
 * on the device, and the outcome (passes, CSTONE_ERR_CAPACITY with the count needed,
 * CSTONE_ERR_NOT_CONVERGED, a timeout) stays in the workspace until cstone_leaves_result reads it.
 * On any failure every set's output is its root array {0, 8^L} (which needs elem_cap >= 2 S), so
 * the phases queued after this call stay within their buffers. */
CSTONE_API int cstone_build_leaves_batched_async(const uint64_t* sorted_keys, int64_t n, const int64_t* set_offsets,
                                                 int32_t n_sets, uint32_t ncrit, uint64_t* elements, int64_t elem_cap,
                                                 int64_t* element_offsets, int32_t warm, uint32_t* counts,
                                                 uint32_t* offsets, int32_t max_iters, void* ws, size_t ws_bytes,
                                                 void* stream);
/* Outcome of the last cstone_build_leaves_batched_async on workspace `ws` (same elem_cap and
 * max_iters): returns its status; *n_elements (host) = elements of the result, or on
 * CSTONE_ERR_CAPACITY the count needed; *iters (host, may be NULL) = passes. Synchronises
 * `stream`. */
CSTONE_API int cstone_leaves_result(void* ws, int64_t elem_cap, int32_t max_iters, void* stream, int64_t* n_elements,
                                    int32_t* iters);

/* Linked octrees of all sets (Sec. 5), concatenated: set s's tree is one breadth-first block of
 * the node arrays, from level_offsets[s][0] to level_offsets[s][22]. All indices (child,
 * level_offsets [S][23], leaf_to_node [n_elements], -1 at end keys) are global node indices.
 * n_nodes = sum over sets of n_l + (n_l - 1) / 7. n_elements and n_nodes may be capacities (upper
 * bounds) instead of the exact counts: the element count is then taken from
 * element_offsets[n_sets] on the device, leaf_to_node is -1 from there to n_elements, and only
 * the exact node count is written. A set whose node count disagrees (input not a cornerstone
 * array) is reported through the workspace error word. Asynchronous. */
CSTONE_API int cstone_link_batched_workspace_size(int64_t n_elements, int32_t n_sets, size_t* bytes);
CSTONE_API int cstone_link_tree_batched(const uint64_t* elements, int64_t n_elements, const int64_t* element_offsets,
                                        int32_t n_sets, int64_t n_nodes, uint64_t* node_keys, int32_t* child,
                                        int32_t* level_offsets, int32_t* leaf_to_node, void* ws, size_t ws_bytes,
                                        void* stream);

/* Node counts of all sets' trees (at most 4096 sets); elem_counts from
 * cstone_build_leaves_batched. n_elements may be the capacity that cstone_link_tree_batched was
 * given (its leaf_to_node is -1 beyond the actual elements). Workspace:
 * cstone_upsweep_workspace_size(1). Asynchronous. */
CSTONE_API int cstone_upsweep_counts_batched(const uint32_t* elem_counts, int64_t n_elements,
                                             const int32_t* leaf_to_node, const int32_t* child,
                                             const int32_t* level_offsets, int32_t n_sets, uint32_t* node_counts,
                                             void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------------------
 * The whole batched build in one call (Sec. 4: the f / g loop of every set from its root, or
 * warm-started from the previous arrays; Sec. 5: the linked octree of every set and its node
 * counts): bounding cubes (when no boxes are given), keys, segmented sort, leaf loop, linked trees
 * and node counts, one launch per phase for all sets. Nothing is read back to the host and nothing
 * is allocated, so the call can be captured in a CUDA graph: the phases after the leaf loop run on
 * the capacities elem_cap and node_cap, the element count of the result is element_offsets[S] and
 * the node count level_offsets[S-1][22] (both on the device), and the outcome stays in the
 * workspace until cstone_build_batched_result reads it. On a failure of the leaf loop (capacity,
 * max_iters, a timeout) every set's output is its root array, so the later phases stay in bounds;
 * the caller then retries with a larger elem_cap (cold, since the warm arrays were overwritten).
 * Per-set results equal those of the single-set calls on each set alone. At most 4096 sets.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    const double* x;             /* [n] float64 device, all sets back to back */
    const double* y;
    const double* z;
    int64_t n;
    const int64_t* set_offsets;  /* [S + 1] int64 device: set s owns particles [off[s], off[s+1]) */
    int32_t n_sets;              /* S, 1 .. 4096 */
    const double* boxes;         /* [S][4] float64 device {lo, side} per set, or NULL: bounding cubes */
} cstone_batch_input;

typedef struct {
    int32_t curve;      /* CSTONE_MORTON or CSTONE_HILBERT */
    uint32_t ncrit;     /* N_crit */
    int32_t max_iters;  /* bound on f / g passes, 1 .. 256 */
    int32_t warm;       /* 0: every set from its root; else elements / element_offsets hold the previous
                           arrays, their element count being element_offsets[S] (on the device) */
} cstone_batch_params;

typedef struct {                /* all device arrays, owned by the caller */
    double* boxes_out;          /* [S][4]: the bounding cubes when input boxes is NULL (else unused) */
    uint64_t* keys;             /* [n] keys in input order */
    uint64_t* sorted_keys;      /* [n] sorted within each set (must not alias keys) */
    uint32_t* perm;             /* [n] global input index of each sorted key */
    uint64_t* elements;         /* [elem_cap] every set's leaves followed by its end key 8^L */
    int64_t elem_cap;           /* at least 2 S */
    int64_t* element_offsets;   /* [S + 1] set s owns elements [eo[s], eo[s+1]) */
    uint32_t* leaf_counts;      /* [elem_cap] (0 at end keys) */
    uint32_t* leaf_offsets;     /* [elem_cap] first sorted particle (global) of each element, or NULL */
    uint64_t* node_keys;        /* [node_cap] NK of every set, one breadth-first block per set */
    int32_t* child;             /* [node_cap] CO, global node indices, 0 for a leaf */
    int32_t* level_offsets;     /* [S][23] LO, global node indices */
    int32_t* leaf_to_node;      /* [elem_cap] global node index of each leaf, -1 at end keys and beyond */
    uint32_t* node_counts;      /* [node_cap] */
    int64_t node_cap;           /* at least elem_cap + elem_cap / 7 + S */
} cstone_batch_buffers;

CSTONE_API int cstone_build_batched_workspace_size(int64_t n, int32_t n_sets, int64_t elem_cap, int32_t max_iters,
                                                   size_t* bytes);
CSTONE_API int cstone_build_batched(const cstone_batch_input* in, const cstone_batch_params* params,
                                    const cstone_batch_buffers* out, void* ws, size_t ws_bytes, void* stream);
/* Outcome of the last cstone_build_batched on `ws` (n, n_sets, elem_cap and max_iters as given to
 * it; level_offsets its output): returns its status, with *n_elements (host) = elements of the
 * result (on CSTONE_ERR_CAPACITY: the count needed), *n_nodes (host) = nodes of all trees and
 * *iters (host, may be NULL) = f / g passes. Synchronises `stream`. */
CSTONE_API int cstone_build_batched_result(const void* ws, int64_t n, int32_t n_sets, int64_t elem_cap,
                                           int32_t max_iters, const int32_t* level_offsets, void* stream,
                                           int64_t* n_elements, int64_t* n_nodes, int32_t* iters);

/* ------------------------------------------------------------------------------------------
 * Full build from host memory (end to end): a particle set's coordinates and masses are copied in
 * from host buffers, the tree is built on the device as by the single-set calls above (bounding
 * cube, keys and multipole records, sort, cornerstone leaves of Sec. 4, linked octree and node
 * counts of Sec. 5, multipoles), and the tree is copied out to host buffers. Two calls per set,
 * so that consecutive sets overlap on the GPU:
 *   cstone_host_stage  copies a set into a device slot (on copy_in_stream);
 *   cstone_host_build  builds a staged slot (on compute_stream) and copies its tree out (on
 *                      copy_out_stream).
 * With two slots, the order stage(0, set 0); for k: { stage((k+1) % 2, set k+1); build(k % 2) }
 * copies set k+1 in while set k builds and set k-1's tree goes out. Host buffers must be pinned
 * (cudaHostAlloc / cudaHostRegister) for the copies to be asynchronous.
 *
 * A slot is caller-owned: a device workspace of cstone_host_workspace_size bytes (256-byte
 * aligned; it holds the staged inputs, every intermediate and output array, and the phases'
 * scratch) and four CUDA events (cudaEvent_t passed as void*, created by the caller, timing may
 * be disabled) through which the calls order the slot's reuse: staged (the set is on the
 * device), inputs_read (the build has read the inputs: the next stage may overwrite them), built
 * (the tree is complete) and copied_out (the tree is on the host: the next build may overwrite
 * it; the caller waits on this event before reading the host tree). A slot must not be staged or
 * built from two host threads at once.
 *
 * cstone_host_build synchronises compute_stream once, after the leaf loop, for the number of
 * leaves; it returns CSTONE_ERR_CAPACITY (with out->n_leaves = the leaves needed) when leaf_cap
 * is too small, and then copies nothing out. Device errors of the phases after the leaf loop are
 * read by cstone_host_status (synchronises compute_stream). n (at least 1), leaf_cap and
 * with_masses must be the values the workspace was sized for.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    void* ws;             /* device workspace, cstone_host_workspace_size bytes */
    size_t ws_bytes;
    void* staged;         /* cudaEvent_t */
    void* inputs_read;    /* cudaEvent_t */
    void* built;          /* cudaEvent_t */
    void* copied_out;     /* cudaEvent_t */
} cstone_host_slot;

typedef struct {              /* host arrays (pinned), owned by the caller; node_cap = leaf_cap + (leaf_cap - 1) / 7 */
    uint64_t* leaves;         /* [leaf_cap + 1] cornerstone array K */
    uint32_t* leaf_counts;    /* [leaf_cap] N_i */
    uint64_t* node_keys;      /* [node_cap] NK */
    int32_t* child;           /* [node_cap] CO */
    int32_t* level_offsets;   /* [23] LO */
    uint32_t* node_counts;    /* [node_cap] */
    float* mass;              /* [node_cap], or NULL without masses */
    double* com;              /* [3 * node_cap]: com[d * n_nodes + i], or NULL */
    float* quad;              /* [6 * node_cap]: quad[q * n_nodes + i] (xx xy xz yy yz zz), or NULL */
    int64_t n_leaves;         /* out (host, set by cstone_host_build) */
    int64_t n_nodes;          /* out */
    int32_t iters;            /* out: f / g passes */
} cstone_host_tree;

CSTONE_API int cstone_host_workspace_size(int64_t n, int64_t leaf_cap, int32_t with_masses, size_t* bytes);
/* hx, hy, hz [n] float64 host; hm [n] float32 host, NULL without masses (then with_masses = 0). */
CSTONE_API int cstone_host_stage(const double* hx, const double* hy, const double* hz, const float* hm, int64_t n,
                                 int64_t leaf_cap, const cstone_host_slot* slot, void* copy_in_stream);
CSTONE_API int cstone_host_build(int64_t n, int64_t leaf_cap, int32_t with_masses, int32_t curve, uint32_t ncrit,
                                 int32_t max_iters, const cstone_host_slot* slot, cstone_host_tree* out,
                                 void* compute_stream, void* copy_out_stream);
/* First device error recorded by the last cstone_host_build on the slot (CSTONE_OK if none). */
CSTONE_API int cstone_host_status(int64_t n, int64_t leaf_cap, int32_t with_masses, const cstone_host_slot* slot,
                                  void* compute_stream);

/* ------------------------------------------------------------------------------------------
 * f and g as separate steps, for a leaf array whose counts are summed over several processes
 * (the global tree of Sec. 6: every rank counts its own particles, the counts are summed by an
 * allreduce, and every rank applies the same g to the summed counts).
 *
 * cstone_leaf_counts (Eq. histogram): counts[i] = number of sorted_keys in [leaves[i],
 *   leaves[i+1]) for i < n_leaves. sorted_keys [n] device, ascending; leaves [n_leaves + 1]
 *   device (a cornerstone array); counts [n_leaves] device output. Asynchronous.
 * cstone_rebalance (Eqs. g1, g2, g3): one pass of the split / merge rule on the given counts,
 *   writing the new array to leaves_out [leaf_cap + 1] (must not alias leaves) with
 *   *n_leaves_out (host) leaves; *changed (host) = 1 if any leaf was split or merged, 0 if the
 *   array is final. Returns CSTONE_ERR_CAPACITY (with *n_leaves_out = the leaves needed) when
 *   the new array does not fit. Synchronises `stream`.
 * ------------------------------------------------------------------------------------------ */
CSTONE_API int cstone_leaf_counts(const uint64_t* sorted_keys, int64_t n, const uint64_t* leaves, int64_t n_leaves,
                                  uint32_t* counts, void* stream);
CSTONE_API int cstone_rebalance_workspace_size(int64_t n_leaves, size_t* bytes);
CSTONE_API int cstone_rebalance(const uint64_t* leaves, const uint32_t* counts, int64_t n_leaves, uint32_t ncrit,
                                uint64_t* leaves_out, int64_t leaf_cap, int64_t* n_leaves_out, int32_t* changed,
                                void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------------------
 * SFC domain decomposition (Sec. 6). A set spread over several processes takes the minimum of the
 * per-axis minima and the maximum of the maxima of cstone_bounds over the processes, and
 * cstone_cube_from_bounds turns them into the bounding cube of the union, with the arithmetic of
 * cstone_bbox: lo = minima, side = largest extent (one IEEE subtraction per axis), side 1 when it is
 * 0 or when there is no point (minima of +inf).
 *   bounds [6] float64 device {min x, min y, min z, max x, max y, max z}; box [4] float64 device
 *   output {lo_x, lo_y, lo_z, side}. Asynchronous.
 *
 * cstone_decompose cuts the globally replicated leaf array into n_ranks bins of consecutive
 * leaves holding about N_tot / n_ranks particles each (the paper's "approximately"; this library's
 * reading): cut r (0 < r < n_ranks) is the first leaf whose preceding leaves hold at least
 * r N_tot / n_ranks particles, compared exactly in integers, n_leaves if no leaf qualifies;
 * cuts[0] = 0, cuts[n_ranks] = n_leaves. Rank r owns leaves [cuts[r], cuts[r+1]), the key range
 * [K[cuts[r]], K[cuts[r+1]]).
 *   counts [n_leaves] uint32 device: the global leaf counts (summed over the processes); their sum
 *          must stay below 2^64 / n_ranks.
 *   n_ranks 1 .. 65536; cuts [n_ranks + 1] int64 device output. Asynchronous.
 * ------------------------------------------------------------------------------------------ */
CSTONE_API int cstone_cube_from_bounds(const double* bounds, double* box, void* stream);
CSTONE_API int cstone_decompose_workspace_size(int64_t n_leaves, int32_t n_ranks, size_t* bytes);
CSTONE_API int cstone_decompose(const uint32_t* counts, int64_t n_leaves, int32_t n_ranks, int64_t* cuts, void* ws,
                                size_t ws_bytes, void* stream);

/* Locally essential octree focused on the key range F = [f_start, f_end) (Sec. 7): one pass of
 * g1^LE, g2, g3 on the given counts. Inside F, and for a node overlapping F, the rule of
 * cstone_rebalance. Outside F a leaf is split only when it also fails the minimum-distance
 * multipole acceptance criterion r_min > l / theta, and 8 sibling leaves are merged when their
 * parent holds at most ncrit particles or lies outside F and passes the criterion. r_min is the
 * smallest distance between the node's cube and the cubes of the maximal octree nodes tiling F,
 * l the node's edge, both in cells of the key grid; the comparison is r_min^2 (an exact integer)
 * > (l / theta)^2 with l / theta and the square each rounded once in IEEE double. An empty F
 * accepts every node. curve: the curve of the keys (their cubes are decoded from them).
 * f_end <= 8^L, theta > 0. Otherwise as cstone_rebalance (same workspace size). Iterating
 * cstone_leaf_counts and this call until *changed == 0 gives the focused tree; on one process the
 * counts are the plain histogram of the process's particles. */
CSTONE_API int cstone_rebalance_focus(const uint64_t* leaves, const uint32_t* counts, int64_t n_leaves, uint32_t ncrit,
                                      uint64_t f_start, uint64_t f_end, double theta, int curve, uint64_t* leaves_out,
                                      int64_t leaf_cap, int64_t* n_leaves_out, int32_t* changed, void* ws,
                                      size_t ws_bytes, void* stream);

/* ==========================================================================================
 * 30-bit keys (L = 10): the other key length of Sec. 3, one 32-bit word per key. Every entry
 * point below is its cstone_* counterpart with uint32_t keys and 10 levels: a key of this
 * family is the top 30 bits of the 63-bit key of the same point (the grid of 2^10 cells per
 * axis nests in the one of 2^21 cells, and both curves nest level by level); end key 8^10 = 2^30;
 * level_offsets has CSTONE30_LEVELS + 2 = 12 entries; the sort takes 4 passes of 8-bit digits;
 * a leaf that is a single level-10 cell is not split whatever its count. Arguments, ownership,
 * errors and synchronisation are those of the 63-bit entry point. The bounding cube
 * (cstone_bbox) does not depend on the key length.
 * ========================================================================================== */
CSTONE_API int cstone30_keys(const double* x, const double* y, const double* z, int64_t n, const double* box,
                             int curve, uint32_t* keys, void* stream);
CSTONE_API int cstone30_sort_workspace_size(int64_t n, size_t* bytes);
CSTONE_API int cstone30_sort(const uint32_t* keys_in, uint32_t* keys_out, uint32_t* perm, int64_t n, void* ws,
                             size_t ws_bytes, void* stream);
CSTONE_API int cstone30_leaves_workspace_size(int64_t n, int64_t leaf_cap, int32_t max_iters, size_t* bytes);
CSTONE_API int cstone30_build_leaves(const uint32_t* sorted_keys, int64_t n, uint32_t ncrit, uint32_t* leaves,
                                     int64_t leaf_cap, int64_t* n_leaves, uint32_t* counts, uint32_t* offsets,
                                     int32_t max_iters, int32_t* iters, void* ws, size_t ws_bytes, void* stream);
CSTONE_API int cstone30_link_workspace_size(int64_t n_leaves, size_t* bytes);
CSTONE_API int cstone30_link_tree(const uint32_t* leaves, int64_t n_leaves, uint32_t* node_keys, int32_t* child,
                                  int32_t* level_offsets, int32_t* leaf_to_node, int32_t* parent, void* ws,
                                  size_t ws_bytes, void* stream);
CSTONE_API int cstone30_upsweep_workspace_size(int64_t n_leaves, size_t* bytes);
CSTONE_API int cstone30_upsweep_counts(const uint32_t* leaf_counts, int64_t n_leaves, const int32_t* leaf_to_node,
                                       const int32_t* child, const int32_t* level_offsets, uint32_t* node_counts,
                                       void* ws, size_t ws_bytes, void* stream);
CSTONE_API int cstone30_multipole_workspace_size(int64_t n, int64_t n_leaves, size_t* bytes);
CSTONE_API int cstone30_leaf_counts(const uint32_t* sorted_keys, int64_t n, const uint32_t* leaves, int64_t n_leaves,
                                    uint32_t* counts, void* stream);
CSTONE_API int cstone30_rebalance_workspace_size(int64_t n_leaves, size_t* bytes);
CSTONE_API int cstone30_rebalance(const uint32_t* leaves, const uint32_t* counts, int64_t n_leaves, uint32_t ncrit,
                                  uint32_t* leaves_out, int64_t leaf_cap, int64_t* n_leaves_out, int32_t* changed,
                                  void* ws, size_t ws_bytes, void* stream);
CSTONE_API int cstone30_rebalance_focus(const uint32_t* leaves, const uint32_t* counts, int64_t n_leaves,
                                        uint32_t ncrit, uint32_t f_start, uint32_t f_end, double theta, int curve,
                                        uint32_t* leaves_out, int64_t leaf_cap, int64_t* n_leaves_out,
                                        int32_t* changed, void* ws, size_t ws_bytes, void* stream);
CSTONE_API int cstone30_upsweep_multipoles(const double* x, const double* y, const double* z, const float* m,
                                           const uint32_t* perm, int64_t n, const uint32_t* offsets, int64_t n_leaves,
                                           const int32_t* leaf_to_node, const int32_t* child,
                                           const int32_t* level_offsets, const double* box, float* mass, double* com,
                                           float* quad, void* ws, size_t ws_bytes, void* stream);
CSTONE_API int cstone30_keys_records(const double* x, const double* y, const double* z, const float* m, int64_t n,
                                     const double* box, int curve, uint32_t* keys, void* records, void* ws,
                                     size_t ws_bytes, void* stream);
CSTONE_API int cstone30_upsweep_multipoles_records(const void* records, const uint32_t* perm, int64_t n,
                                                   const uint32_t* offsets, int64_t n_leaves,
                                                   const int32_t* leaf_to_node, const int32_t* child,
                                                   const int32_t* level_offsets, const double* box, float* mass,
                                                   double* com, float* quad, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CSTONE_H */
