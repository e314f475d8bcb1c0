// Full build from host memory (end to end): a particle set is copied into a caller-owned device
// slot, built there by the single-set calls (bounding cube, keys with the multipole records, sort,
// the cornerstone leaf loop of Sec. 4, the linked octree and node counts of Sec. 5, the multipole
// upsweep), and its tree is copied back to host memory. Staging and building are separate calls,
// so that with two slots the copy-in of one set runs while the previous set builds and the one
// before it is copied out; four caller-created events per slot order the reuse of its memory.
// 63-bit keys only. Host code only: every step runs in the library's kernels.
#ifndef CSTONE_KEY32
#include "common.cuh"

namespace cst {
namespace {

// The slot's device memory: the staged inputs, every array of the build, and one scratch
// workspace per phase (each keeps its own error word).
enum {
    kX, kY, kZ, kM, kBox, kKeys, kSorted, kPerm, kRec, kLeaves, kCounts, kOffsets, kNK, kCO, kLO, kL2N, kParent,
    kNCounts, kMass, kCom, kQuad, kWsBbox, kWsRec, kWsSort, kWsLeaves, kWsLink, kWsCounts, kWsMp, kParts
};
constexpr int kMaxItersSized = 256;  // the leaf workspace does not depend on max_iters

struct HostLayout {
    size_t off[kParts];
    size_t len[kParts];
    size_t bytes;
    int64_t node_cap;
};

constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }

int host_layout(int64_t n, int64_t cap, bool masses, HostLayout* l) {
    const size_t N = static_cast<size_t>(n), C = static_cast<size_t>(cap);
    const int64_t nc = cap + (cap - 1) / 7;
    const size_t NC = static_cast<size_t>(nc);
    size_t len[kParts] = {};
    len[kX] = len[kY] = len[kZ] = 8 * N;
    len[kM] = 4 * N;  // reserved with or without masses: the staged inputs sit at the same offsets either way
    len[kBox] = 4 * sizeof(double);
    len[kKeys] = len[kSorted] = 8 * N;
    len[kPerm] = 4 * N;
    if (masses)
        if (int rc = cstone_records_size(n, &len[kRec])) return rc;
    len[kLeaves] = 8 * (C + 1);
    len[kCounts] = 4 * C;
    len[kOffsets] = 4 * (C + 1);
    len[kNK] = 8 * NC;
    len[kCO] = 4 * NC;
    len[kLO] = 4 * (CSTONE_LEVELS + 2);
    len[kL2N] = 4 * C;
    len[kParent] = 4 * (NC / 8 + 1);
    len[kNCounts] = 4 * NC;
    len[kMass] = masses ? 4 * NC : 0;
    len[kCom] = masses ? 3 * 8 * NC : 0;
    len[kQuad] = masses ? 6 * 4 * NC : 0;
    if (int rc = cstone_bbox_workspace_size(n, &len[kWsBbox])) return rc;
    if (masses)
        if (int rc = cstone_keys_records_workspace_size(&len[kWsRec])) return rc;
    if (int rc = cstone_sort_workspace_size(n, &len[kWsSort])) return rc;
    if (int rc = cstone_leaves_workspace_size(n, cap, kMaxItersSized, &len[kWsLeaves])) return rc;
    if (int rc = cstone_link_workspace_size(cap, &len[kWsLink])) return rc;
    if (int rc = cstone_upsweep_workspace_size(cap, &len[kWsCounts])) return rc;
    if (masses)
        if (int rc = cstone_multipole_workspace_size(0, cap, &len[kWsMp])) return rc;
    size_t off = 0;
    for (int k = 0; k < kParts; ++k) {
        l->off[k] = off;
        l->len[k] = round256(len[k]);
        off += l->len[k];
    }
    l->bytes = off;
    l->node_cap = nc;
    return CSTONE_OK;
}

int check_args(int64_t n, int64_t cap, const cstone_host_slot* slot, const char* who) {
    if (n < 1 || n >= CSTONE_MAX_PARTICLES || cap < 1 || cap > CSTONE_MAX_LEAVES || !slot || !slot->ws ||
        !slot->staged || !slot->inputs_read || !slot->built || !slot->copied_out)
        return fail(CSTONE_ERR_INVALID_ARG, "%s: bad argument (n=%lld, leaf_cap=%lld, slot and its events non-NULL)",
                    who, (long long)n, (long long)cap);
    return CSTONE_OK;
}

cudaEvent_t ev(void* e) { return static_cast<cudaEvent_t>(e); }

}  // namespace
}  // namespace cst

extern "C" {

int cstone_host_workspace_size(int64_t n, int64_t leaf_cap, int32_t with_masses, size_t* bytes) {
    if (!bytes || n < 1 || n >= CSTONE_MAX_PARTICLES || leaf_cap < 1 || leaf_cap > CSTONE_MAX_LEAVES)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_host_workspace_size: bad argument");
    cst::HostLayout l;
    if (int rc = cst::host_layout(n, leaf_cap, with_masses != 0, &l)) return rc;
    *bytes = l.bytes;
    return CSTONE_OK;
}

int cstone_host_stage(const double* hx, const double* hy, const double* hz, const float* hm, int64_t n,
                      int64_t leaf_cap, const cstone_host_slot* slot, void* copy_in_stream) {
    if (int rc = cst::check_args(n, leaf_cap, slot, "cstone_host_stage")) return rc;
    if (!hx || !hy || !hz)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_host_stage: NULL coordinates");
    cst::HostLayout l;
    if (int rc = cst::host_layout(n, leaf_cap, hm != nullptr, &l)) return rc;
    if (int rc = cst::check_ws(slot->ws, slot->ws_bytes, l.bytes, "cstone_host_stage")) return rc;
    char* base = static_cast<char*>(slot->ws);
    const cudaStream_t st = cst::as_stream(copy_in_stream);
    // the slot's previous build has read its inputs
    CST_CUDA(cudaStreamWaitEvent(st, cst::ev(slot->inputs_read), 0));
    const size_t b8 = 8 * static_cast<size_t>(n);
    CST_CUDA(cudaMemcpyAsync(base + l.off[cst::kX], hx, b8, cudaMemcpyHostToDevice, st));
    CST_CUDA(cudaMemcpyAsync(base + l.off[cst::kY], hy, b8, cudaMemcpyHostToDevice, st));
    CST_CUDA(cudaMemcpyAsync(base + l.off[cst::kZ], hz, b8, cudaMemcpyHostToDevice, st));
    if (hm) CST_CUDA(cudaMemcpyAsync(base + l.off[cst::kM], hm, 4 * static_cast<size_t>(n), cudaMemcpyHostToDevice, st));
    CST_CUDA(cudaEventRecord(cst::ev(slot->staged), st));
    return CSTONE_OK;
}

int cstone_host_build(int64_t n, int64_t leaf_cap, int32_t with_masses, int32_t curve, uint32_t ncrit,
                      int32_t max_iters, const cstone_host_slot* slot, cstone_host_tree* out, void* compute_stream,
                      void* copy_out_stream) {
    if (int rc = cst::check_args(n, leaf_cap, slot, "cstone_host_build")) return rc;
    const bool masses = with_masses != 0;
    if (!out || !out->leaves || !out->leaf_counts || !out->node_keys || !out->child || !out->level_offsets ||
        !out->node_counts || (masses && (!out->mass || !out->com || !out->quad)) ||
        (curve != CSTONE_MORTON && curve != CSTONE_HILBERT) || max_iters < 1 || max_iters > 256)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_host_build: bad output arrays or parameters");
    cst::HostLayout l;
    if (int rc = cst::host_layout(n, leaf_cap, masses, &l)) return rc;
    if (int rc = cst::check_ws(slot->ws, slot->ws_bytes, l.bytes, "cstone_host_build")) return rc;
    char* base = static_cast<char*>(slot->ws);
    auto at = [&](int k) { return static_cast<void*>(base + l.off[k]); };
    auto ws = [&](int k) { return at(k); };
    const cudaStream_t st = cst::as_stream(compute_stream), so = cst::as_stream(copy_out_stream);
    const double* x = static_cast<const double*>(at(cst::kX));
    const double* y = static_cast<const double*>(at(cst::kY));
    const double* z = static_cast<const double*>(at(cst::kZ));
    double* box = static_cast<double*>(at(cst::kBox));
    uint64_t* keys = static_cast<uint64_t*>(at(cst::kKeys));
    uint64_t* sorted = static_cast<uint64_t*>(at(cst::kSorted));
    uint32_t* perm = static_cast<uint32_t*>(at(cst::kPerm));
    uint64_t* leaves = static_cast<uint64_t*>(at(cst::kLeaves));
    uint32_t* counts = static_cast<uint32_t*>(at(cst::kCounts));
    uint32_t* offsets = static_cast<uint32_t*>(at(cst::kOffsets));
    uint64_t* nk = static_cast<uint64_t*>(at(cst::kNK));
    int32_t* co = static_cast<int32_t*>(at(cst::kCO));
    int32_t* lo = static_cast<int32_t*>(at(cst::kLO));
    int32_t* l2n = static_cast<int32_t*>(at(cst::kL2N));
    int32_t* parent = static_cast<int32_t*>(at(cst::kParent));
    uint32_t* ncounts = static_cast<uint32_t*>(at(cst::kNCounts));

    // the set is on the device, and the slot's previous tree has been copied out
    CST_CUDA(cudaStreamWaitEvent(st, cst::ev(slot->staged), 0));
    CST_CUDA(cudaStreamWaitEvent(st, cst::ev(slot->copied_out), 0));
    if (int rc = cstone_bbox(x, y, z, n, box, ws(cst::kWsBbox), l.len[cst::kWsBbox], st)) return rc;
    if (masses) {
        if (int rc = cstone_keys_records(x, y, z, static_cast<const float*>(at(cst::kM)), n, box, curve, keys,
                                         at(cst::kRec), ws(cst::kWsRec), l.len[cst::kWsRec], st))
            return rc;
    } else if (int rc = cstone_keys(x, y, z, n, box, curve, keys, st)) {
        return rc;
    }
    CST_CUDA(cudaEventRecord(cst::ev(slot->inputs_read), st));  // the next stage may overwrite x, y, z, m
    if (int rc = cstone_sort(keys, sorted, perm, n, ws(cst::kWsSort), l.len[cst::kWsSort], st)) return rc;
    int64_t nl = 0;
    int32_t iters = 0;
    const int rc_leaves = cstone_build_leaves(sorted, n, ncrit, leaves, leaf_cap, &nl, counts, offsets, max_iters,
                                              &iters, ws(cst::kWsLeaves), l.len[cst::kWsLeaves], st);
    out->n_leaves = nl;
    out->iters = iters;
    out->n_nodes = 0;
    if (rc_leaves) return rc_leaves;
    const int64_t nn = nl + (nl - 1) / 7;
    out->n_nodes = nn;
    if (int rc = cstone_link_tree(leaves, nl, nk, co, lo, l2n, parent, ws(cst::kWsLink), l.len[cst::kWsLink], st))
        return rc;
    if (int rc = cstone_upsweep_counts(counts, nl, l2n, co, lo, ncounts, ws(cst::kWsCounts), l.len[cst::kWsCounts],
                                       st))
        return rc;
    float* mass = static_cast<float*>(at(cst::kMass));
    double* com = static_cast<double*>(at(cst::kCom));
    float* quad = static_cast<float*>(at(cst::kQuad));
    if (masses) {
        if (int rc = cstone_upsweep_multipoles_records(at(cst::kRec), perm, n, offsets, nl, l2n, co, lo, box, mass,
                                                       com, quad, ws(cst::kWsMp), l.len[cst::kWsMp], st))
            return rc;
    }
    CST_CUDA(cudaEventRecord(cst::ev(slot->built), st));

    // the tree out, sized to the built tree
    CST_CUDA(cudaStreamWaitEvent(so, cst::ev(slot->built), 0));
    const size_t L1 = static_cast<size_t>(nl), NN = static_cast<size_t>(nn);
    CST_CUDA(cudaMemcpyAsync(out->leaves, leaves, 8 * (L1 + 1), cudaMemcpyDeviceToHost, so));
    CST_CUDA(cudaMemcpyAsync(out->leaf_counts, counts, 4 * L1, cudaMemcpyDeviceToHost, so));
    CST_CUDA(cudaMemcpyAsync(out->node_keys, nk, 8 * NN, cudaMemcpyDeviceToHost, so));
    CST_CUDA(cudaMemcpyAsync(out->child, co, 4 * NN, cudaMemcpyDeviceToHost, so));
    CST_CUDA(cudaMemcpyAsync(out->level_offsets, lo, 4 * (CSTONE_LEVELS + 2), cudaMemcpyDeviceToHost, so));
    CST_CUDA(cudaMemcpyAsync(out->node_counts, ncounts, 4 * NN, cudaMemcpyDeviceToHost, so));
    if (masses) {
        CST_CUDA(cudaMemcpyAsync(out->mass, mass, 4 * NN, cudaMemcpyDeviceToHost, so));
        CST_CUDA(cudaMemcpyAsync(out->com, com, 3 * 8 * NN, cudaMemcpyDeviceToHost, so));
        CST_CUDA(cudaMemcpyAsync(out->quad, quad, 6 * 4 * NN, cudaMemcpyDeviceToHost, so));
    }
    CST_CUDA(cudaEventRecord(cst::ev(slot->copied_out), so));
    return CSTONE_OK;
}

int cstone_host_status(int64_t n, int64_t leaf_cap, int32_t with_masses, const cstone_host_slot* slot,
                       void* compute_stream) {
    if (int rc = cst::check_args(n, leaf_cap, slot, "cstone_host_status")) return rc;
    cst::HostLayout l;
    if (int rc = cst::host_layout(n, leaf_cap, with_masses != 0, &l)) return rc;
    if (int rc = cst::check_ws(slot->ws, slot->ws_bytes, l.bytes, "cstone_host_status")) return rc;
    const char* base = static_cast<const char*>(slot->ws);
    // the phases that record device errors in their workspace header (the bounding cube records none)
    const int parts[] = {cst::kWsRec, cst::kWsSort, cst::kWsLink, cst::kWsCounts, cst::kWsMp};
    for (int k : parts) {
        if (l.len[k] == 0) continue;
        int status = 0;
        if (int rc = cstone_workspace_status(base + l.off[k], compute_stream, &status)) return rc;
        if (status) return cst::fail(status, "cstone_host_build: device error in phase workspace %d", k);
    }
    return CSTONE_OK;
}

}  // extern "C"
#endif
