// The batched build as one call: bounding cubes (optional), keys, segmented sort, the cornerstone
// leaf loop of every set (Sec. 4), the linked octrees (Sec. 5) and their node counts, one launch
// (or one cooperative launch) per phase for all sets, with no host synchronisation: the phases run
// on capacities, the element and node counts stay on the device, and the outcome stays in the
// workspace until cstone_build_batched_result reads it. 63-bit keys only.
#ifndef CSTONE_KEY32
#include "common.cuh"

namespace cst {
namespace {

// The workspace: this call's header, then one workspace per phase (each keeps its own error word).
enum { kWsKeys, kWsSort, kWsLeaves, kWsLink, kWsCounts, kWsParts };

struct BuildLayout {
    size_t off[kWsParts];
    size_t len[kWsParts];
    size_t bytes;
};

constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }

int build_layout(int64_t n, int32_t n_sets, int64_t elem_cap, int32_t max_iters, BuildLayout* l) {
    size_t len[kWsParts];
    if (int rc = cstone_keys_batched_workspace_size(n_sets, &len[kWsKeys])) return rc;
    if (int rc = cstone_sort_segmented_workspace_size(n, n_sets, &len[kWsSort])) return rc;
    if (int rc = cstone_leaves_batched_workspace_size(elem_cap, max_iters, &len[kWsLeaves])) return rc;
    if (int rc = cstone_link_batched_workspace_size(elem_cap, n_sets, &len[kWsLink])) return rc;
    if (int rc = cstone_upsweep_workspace_size(1, &len[kWsCounts])) return rc;
    size_t off = sizeof(WsHeader);
    for (int k = 0; k < kWsParts; ++k) {
        l->off[k] = off;
        l->len[k] = round256(len[k]);
        off += l->len[k];
    }
    l->bytes = off;
    return CSTONE_OK;
}

constexpr int kMaxSets = 4096;  // the batched count upsweep's limit

}  // namespace
}  // namespace cst

extern "C" {

int cstone_build_batched_workspace_size(int64_t n, int32_t n_sets, int64_t elem_cap, int32_t max_iters,
                                        size_t* bytes) {
    if (!bytes || n < 0 || n >= CSTONE_MAX_PARTICLES || n_sets < 1 || n_sets > cst::kMaxSets ||
        elem_cap < 2 * (int64_t)n_sets || elem_cap > CSTONE_MAX_LEAVES || max_iters < 1 || max_iters > 256)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_batched_workspace_size: bad argument");
    cst::BuildLayout l;
    if (int rc = cst::build_layout(n, n_sets, elem_cap, max_iters, &l)) return rc;
    *bytes = l.bytes;
    return CSTONE_OK;
}

int cstone_build_batched(const cstone_batch_input* in, const cstone_batch_params* prm,
                         const cstone_batch_buffers* out, void* ws, size_t ws_bytes, void* stream) {
    if (!in || !prm || !out)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_batched: NULL input, parameters or buffers");
    const int64_t n = in->n;
    const int32_t S = in->n_sets;
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || S < 1 || S > cst::kMaxSets || !in->set_offsets ||
        (n > 0 && (!in->x || !in->y || !in->z)) || (!in->boxes && !out->boxes_out))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_batched: bad input (n=%lld, sets=%d)", (long long)n, S);
    if ((prm->curve != CSTONE_MORTON && prm->curve != CSTONE_HILBERT) || prm->max_iters < 1 || prm->max_iters > 256)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_batched: bad parameters (curve %d, max_iters %d)",
                         prm->curve, prm->max_iters);
    const int64_t ecap = out->elem_cap;
    if (ecap < 2 * (int64_t)S || ecap > CSTONE_MAX_LEAVES || out->node_cap < ecap + ecap / 7 + S)
        return cst::fail(CSTONE_ERR_INVALID_ARG,
                         "cstone_build_batched: elem_cap %lld (at least 2 S) or node_cap %lld (at least elem_cap + "
                         "elem_cap / 7 + S) too small",
                         (long long)ecap, (long long)out->node_cap);
    if (!out->keys || !out->sorted_keys || !out->perm || out->keys == out->sorted_keys || !out->elements ||
        !out->element_offsets || !out->leaf_counts || !out->node_keys || !out->child || !out->level_offsets ||
        !out->leaf_to_node || !out->node_counts)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_batched: missing (or aliased key) output buffer");
    cst::BuildLayout l;
    if (int rc = cst::build_layout(n, S, ecap, prm->max_iters, &l)) return rc;
    if (int rc = cst::check_ws(ws, ws_bytes, l.bytes, "cstone_build_batched")) return rc;
    char* base = static_cast<char*>(ws);
    auto part = [&](int k) { return static_cast<void*>(base + l.off[k]); };
    CST_CUDA(cudaMemsetAsync(ws, 0, sizeof(cst::WsHeader), cst::as_stream(stream)));

    const double* boxes = in->boxes;
    if (!boxes) {
        if (int rc = cstone_bbox_batched(in->x, in->y, in->z, in->set_offsets, S, out->boxes_out, stream)) return rc;
        boxes = out->boxes_out;
    }
    if (int rc = cstone_keys_batched(in->x, in->y, in->z, n, in->set_offsets, S, boxes, prm->curve, out->keys,
                                     part(cst::kWsKeys), l.len[cst::kWsKeys], stream))
        return rc;
    if (int rc = cstone_sort_segmented(out->keys, out->sorted_keys, out->perm, n, in->set_offsets, S,
                                       part(cst::kWsSort), l.len[cst::kWsSort], stream))
        return rc;
    if (int rc = cstone_build_leaves_batched_async(out->sorted_keys, n, in->set_offsets, S, prm->ncrit, out->elements,
                                                   ecap, out->element_offsets, prm->warm ? 1 : 0, out->leaf_counts,
                                                   out->leaf_offsets, prm->max_iters, part(cst::kWsLeaves),
                                                   l.len[cst::kWsLeaves], stream))
        return rc;
    if (int rc = cstone_link_tree_batched(out->elements, ecap, out->element_offsets, S, out->node_cap, out->node_keys,
                                          out->child, out->level_offsets, out->leaf_to_node, part(cst::kWsLink),
                                          l.len[cst::kWsLink], stream))
        return rc;
    return cstone_upsweep_counts_batched(out->leaf_counts, ecap, out->leaf_to_node, out->child, out->level_offsets, S,
                                         out->node_counts, part(cst::kWsCounts), l.len[cst::kWsCounts], stream);
}

int cstone_build_batched_result(const void* ws, int64_t n, int32_t n_sets, int64_t elem_cap, int32_t max_iters,
                                const int32_t* level_offsets, void* stream, int64_t* n_elements, int64_t* n_nodes,
                                int32_t* iters) {
    if (!ws || !level_offsets || !n_elements || !n_nodes)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_batched_result: bad argument");
    cst::BuildLayout l;
    if (int rc = cst::build_layout(n, n_sets, elem_cap, max_iters, &l)) return rc;
    const char* base = static_cast<const char*>(ws);
    // the leaf loop first: its status carries the capacity needed on an overflow
    int64_t ne = 0;
    int32_t it = 0;
    int rc = cstone_leaves_result(const_cast<char*>(base) + l.off[cst::kWsLeaves], elem_cap, max_iters, stream, &ne,
                                  &it);
    *n_elements = ne;
    if (iters) *iters = it;
    if (rc) return rc;
    // the device error words of the phases that record device errors, and the node count, in one
    // read-back
    cudaStream_t st = cst::as_stream(stream);
    constexpr int kChecked = 3;
    cst::WsHeader h[kChecked];
    const int parts[kChecked] = {cst::kWsSort, cst::kWsLink, cst::kWsCounts};
    const char* names[kChecked] = {"segmented sort", "link", "node counts"};
    for (int k = 0; k < kChecked; ++k)
        CST_CUDA(cudaMemcpyAsync(&h[k], base + l.off[parts[k]], sizeof(cst::WsHeader), cudaMemcpyDeviceToHost, st));
    int32_t nn = 0;
    CST_CUDA(cudaMemcpyAsync(&nn, level_offsets + (size_t)n_sets * (CSTONE_LEVELS + 2) - 1, sizeof(int32_t),
                             cudaMemcpyDeviceToHost, st));
    CST_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < kChecked; ++k)
        if (h[k].err)
            return cst::fail(static_cast<int>(h[k].err), "cstone_build_batched: %s phase: device error %u (info 0x%x)",
                             names[k], h[k].err, h[k].err_info);
    *n_nodes = nn;
    return CSTONE_OK;
}

}  // extern "C"
#endif
