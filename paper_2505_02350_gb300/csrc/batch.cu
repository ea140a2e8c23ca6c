// Many fields advanced together: one Algorithm 3 epoch of every field of a
// batch in a fixed number of launches, whatever the number of fields.  The
// fused forward + adjoint of all fields is ONE persistent launch whose blocks
// claim (field, work item) pairs from a single counter; the neighbour
// rebuild, the finishing reductions, the optimiser step, the deletion and
// the addition run one launch per stage with a grid row per field.  Every
// field keeps its own buffers and workspace, and the arithmetic of each
// field is the single-field arithmetic, so a field advanced in a batch gets
// the same bits as when it is advanced alone with the same warps per item.
#include <string.h>

#include <vector>

#include "common.cuh"

namespace serbf {
size_t fwd_args_size();
size_t finish_args_size();
int batch_forward_args(const serbf_points *, const serbf_params *, const serbf_config *, float *, float *, uint8_t *,
                       float *, double *, serbf_workspace *, void *, void *, int64_t *);
int batch_pick_warps(int64_t nitems, int sm_count, int fixed);
int batch_forward_launch(const void *args, const void *fin, const uint32_t *item_off, int nfields, uint32_t *counters,
                         int64_t total_items, int64_t finish_blocks, int G, int kahan, int sm_count, cudaStream_t s);
size_t rebuild_args_size();
int batch_rebuild_args(const serbf_points *, const serbf_params *, const serbf_config *, serbf_workspace *, void *,
                       int *, int64_t *, int *, int *);
int batch_rebuild_launch(const void *args, int nfields, int level1_blocks, int64_t chunks, int nsuper, int two_level,
                         cudaStream_t s);
size_t step_args_size();
int batch_step_args(serbf_params *, const float *, float *, float *, serbf_state *, double *, const serbf_config *,
                    serbf_workspace *, void *, int *);
int batch_step_launch(const void *args, int nfields, int max_nb, cudaStream_t s);
size_t add_args_size();
int batch_add_args(const serbf_points *, const float *, const float *, const uint8_t *, serbf_params *, float *,
                   float *, serbf_state *, const double *, const serbf_config *, serbf_workspace *, void *);
int batch_add_launch(const void *args, int nfields, int sm_count, cudaStream_t s);
}  // namespace serbf

using namespace serbf;

namespace {
constexpr uint64_t kBatchMagic = 0x53455242464241ull;  // "SERBFBA"
constexpr int kMaxFields = 1024;

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Device layout of the batch tables, in this order, each 256-byte aligned.
struct Layout {
    size_t fwd, fin, reb, step, add, off, ctr, total;
};

Layout layout(int n) {
    Layout L;
    size_t o = 0;
    L.fwd = o;
    o = up256(o + (size_t)n * fwd_args_size());
    L.fin = o;
    o = up256(o + (size_t)n * finish_args_size());
    L.reb = o;
    o = up256(o + (size_t)n * rebuild_args_size());
    L.step = o;
    o = up256(o + (size_t)n * step_args_size());
    L.add = o;
    o = up256(o + (size_t)n * add_args_size());
    L.off = o;
    o = up256(o + (size_t)(n + 1) * sizeof(uint32_t));
    L.ctr = o;
    o = up256(o + 16 * sizeof(uint32_t));
    L.total = o;
    return L;
}
}  // namespace

struct serbf_batch {
    uint64_t magic;
    int32_t nfields;
    int32_t G, kahan, sm_count;
    char *base;
    Layout L;
    int64_t total_items, finish_blocks, chunks;
    int32_t level1_blocks, nsuper, two_level, step_nb;
};

extern "C" {

size_t serbf_batch_struct_size(void) { return sizeof(serbf_batch); }

int serbf_batch_bytes(int32_t nfields, size_t *bytes) {
    if (nfields < 1 || nfields > kMaxFields || !bytes) return SERBF_EINVAL;
    *bytes = layout(nfields).total;
    return SERBF_OK;
}

int serbf_batch_init(serbf_batch *b, const serbf_field *fields, int32_t nfields, int32_t fwd_warps, void *dev,
                     size_t bytes, void *stream) {
    SERBF_TRACE();
    if (!b || !fields || nfields < 1 || nfields > kMaxFields || !dev || ((uintptr_t)dev) % 256) return SERBF_EINVAL;
    if (fwd_warps != 0 && fwd_warps != 1 && fwd_warps != 2 && fwd_warps != 4 && fwd_warps != 8) return SERBF_EINVAL;
    const Layout L = layout(nfields);
    if (bytes < L.total) return SERBF_ENOMEM;
    std::vector<char> host(L.total, 0);
    int64_t total = 0, fin_blocks = 1, chunks = 0;
    int lvl1 = 1, nsup = 1, two = 0, step_nb = 1, sm = 0;
    const int kahan = fields[0].cfg ? fields[0].cfg->kahan : 0;
    uint32_t *off = reinterpret_cast<uint32_t *>(host.data() + L.off);
    for (int f = 0; f < nfields; ++f) {
        const serbf_field &F = fields[f];
        if (!F.cfg || !F.ws || F.ws->magic != kMagic || !F.ws->binned || F.cfg->kahan != kahan) return SERBF_EINVAL;
        serbf_params prm = F.prm;
        int64_t fb = 1, ch = 0;
        int l1 = 0, ns = 0, tw = 0, nb = 0;
        int rc = batch_forward_args(&F.pts, &F.prm, F.cfg, F.psi, F.err, F.mask, F.grad, F.stats, F.ws,
                                    host.data() + L.fwd + (size_t)f * fwd_args_size(),
                                    host.data() + L.fin + (size_t)f * finish_args_size(), &fb);
        if (!rc) rc = batch_rebuild_args(&F.pts, &F.prm, F.cfg, F.ws, host.data() + L.reb + (size_t)f * rebuild_args_size(),
                                         &l1, &ch, &ns, &tw);
        if (!rc) rc = batch_step_args(&prm, F.grad, F.adam_m, F.adam_v, F.st, F.stats, F.cfg, F.ws,
                                      host.data() + L.step + (size_t)f * step_args_size(), &nb);
        if (!rc) rc = batch_add_args(&F.pts, F.S_raw, F.err, F.mask, &prm, F.adam_m, F.adam_v, F.st, F.stats, F.cfg,
                                     F.ws, host.data() + L.add + (size_t)f * add_args_size());
        if (rc) return rc;
        if (!F.grad) return SERBF_EINVAL;
        off[f] = (uint32_t)total;
        total += F.ws->nitems;
        if (total >= (int64_t)1 << 32) return SERBF_ECAPACITY;
        fin_blocks = fb > fin_blocks ? fb : fin_blocks;
        chunks = ch > chunks ? ch : chunks;
        lvl1 = l1 > lvl1 ? l1 : lvl1;
        nsup = ns > nsup ? ns : nsup;
        two |= tw;
        step_nb = nb > step_nb ? nb : step_nb;
        sm = F.ws->sm_count;
    }
    off[nfields] = (uint32_t)total;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(dev, host.data(), L.total, cudaMemcpyHostToDevice, s) != cudaSuccess) return SERBF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    memset(b, 0, sizeof(*b));
    b->magic = kBatchMagic;
    b->nfields = nfields;
    b->G = batch_pick_warps(total, sm, fwd_warps);
    b->kahan = kahan;
    b->sm_count = sm;
    b->base = static_cast<char *>(dev);
    b->L = L;
    b->total_items = total;
    b->finish_blocks = fin_blocks;
    b->chunks = chunks;
    b->level1_blocks = lvl1;
    b->nsuper = nsup;
    b->two_level = two;
    b->step_nb = step_nb;
    return SERBF_OK;
}

int serbf_batch_warps(const serbf_batch *b) { return (b && b->magic == kBatchMagic) ? b->G : SERBF_EINVAL; }

int serbf_epoch_batched(serbf_batch *b, void *stream) {
    SERBF_TRACE();
    if (!b || b->magic != kBatchMagic) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    char *d = b->base;
    int rc = batch_rebuild_launch(d + b->L.reb, b->nfields, b->level1_blocks, b->chunks, b->nsuper, b->two_level, s);
    if (!rc)
        rc = batch_forward_launch(d + b->L.fwd, d + b->L.fin, reinterpret_cast<const uint32_t *>(d + b->L.off),
                                  b->nfields, reinterpret_cast<uint32_t *>(d + b->L.ctr), b->total_items,
                                  b->finish_blocks, b->G, b->kahan, b->sm_count, s);
    if (!rc) rc = batch_step_launch(d + b->L.step, b->nfields, b->step_nb, s);
    if (!rc) rc = batch_add_launch(d + b->L.add, b->nfields, b->sm_count, s);
    return rc;
}

}  // extern "C"
