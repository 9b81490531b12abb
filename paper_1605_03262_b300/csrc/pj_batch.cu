// Batched form: one persistent launch over several (model, state batch) items of uneven size.
//
// pj_batch_create builds a plan once: per item the group width (the model's configured warps per
// state, halved while one state does not fit next to the kernel's own shared memory) and the
// number of groups a CTA runs for it (limited by shared memory), and a tile list
// (consecutive states of one item) ordered with the costliest tiles first. The plan's device
// memory holds the item table, the tiles and a tile counter. pj_batch_run zeroes the counter and
// launches the persistent kernel on the caller's stream; it allocates nothing and does not
// synchronise, so the pair can be captured into a CUDA graph and replayed as long as the item
// buffers stay where they were when the plan was built.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pyjac_b300.h"
#include "pj_internal.h"

namespace {

int bfail(int code, const std::string &msg) { return pj::set_error(code, msg); }

int bcuda(cudaError_t e, const char *what) {
    return bfail(PJ_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

int check_dev(const void *p, int dev, const char *name) {
    if (!p) return bfail(PJ_EINVAL, std::string(name) + " is NULL");
    if (reinterpret_cast<uintptr_t>(p) & 7) return bfail(PJ_EINVAL, std::string(name) + " is not 8-byte aligned");
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return bfail(PJ_EINVAL, std::string(name) + " is not a CUDA-accessible pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return bfail(PJ_EINVAL, std::string(name) + " is not a device pointer");
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return bfail(PJ_EINVAL, std::string(name) + " lives on another device");
    return PJ_OK;
}

}  // namespace

extern "C" {

int pj_batch_create(const pj_batch_item *items, int n_items, int which, const pj_batch_shape *shape, pj_batch **out) {
    return pj_batch_create_ex(items, n_items, which, shape, nullptr, out);
}

int pj_batch_create_ex(const pj_batch_item *items, int n_items, int which, const pj_batch_shape *shape,
                       const pj_batch_item_shape *item_shapes, pj_batch **out) {
    if (!items || n_items < 1 || !out || (which != 0 && which != 1))
        return bfail(PJ_EINVAL, "pj_batch_create: bad argument");
    *out = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bcuda(e, "cudaGetDevice");
    int sms = 0, optin = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const bool jac = which == 0;
    size_t static_smem = 0;
    if ((e = pj::prepare_batch_kernel(jac, 0, &static_smem)) != cudaSuccess) return bcuda(e, "batch kernel attributes");
    const size_t budget = size_t(optin) > static_smem ? size_t(optin) - static_smem : 0;

    int threads = shape && shape->threads_per_cta > 0 ? shape->threads_per_cta : 512;
    const int ctas = shape && shape->ctas_per_sm > 0 ? shape->ctas_per_sm : 1;
    const int tile_req = shape ? shape->tile_states : 0;
    if (threads % 32 || threads < 32 || threads > 512 || ctas > 32 || tile_req < 0)
        return bfail(PJ_EINVAL, "pj_batch_create: shape outside the supported limits");

    std::vector<pj::BatchItem> bi(n_items);
    std::vector<double> cost(n_items);
    size_t smem = 0;
    for (int i = 0; i < n_items; ++i) {
        const pj_batch_item &it = items[i];
        const pj_mech *m = it.mech;
        if (!m || it.n < 0) return bfail(PJ_EINVAL, "pj_batch_create: item " + std::to_string(i) + ": null model or n < 0");
        if (m->device != dev) return bfail(PJ_EINVAL, "pj_batch_create: item model lives on another device");
        const int64_t N = m->N, nn = (N + 1) * (N + 1);
        if (it.ldy < N || (jac && it.ldj < nn) || ((!jac || it.dydt) && it.ldd < N + 1))
            return bfail(PJ_EINVAL, "pj_batch_create: item " + std::to_string(i) + ": leading dimension too small");
        int rc;
        if (it.n > 0) {
            if ((rc = check_dev(it.T, dev, "T")) || (rc = check_dev(it.P, dev, "P")) || (rc = check_dev(it.Y, dev, "Y")))
                return rc;
            if (jac && (rc = check_dev(it.jac, dev, "jac"))) return rc;
            if ((!jac || it.dydt) && (rc = check_dev(it.dydt, dev, "dydt"))) return rc;
        }
        int wps = 0, groups = 0;
        pj::Scratch sc{};
        const pj_batch_item_shape *is = item_shapes ? &item_shapes[i] : nullptr;
        if (is && (is->warps_per_state < 0 || is->states_per_cta < 0 || is->tile_states < 0))
            return bfail(PJ_EINVAL, "pj_batch_create: item " + std::to_string(i) + ": negative shape entry");
        if (is && is->warps_per_state > 0) {
            // the caller's group width and (optionally) states per CTA, checked against the CTA
            wps = is->warps_per_state;
            if (!(wps == 1 || wps == 2 || wps == 4 || wps == 8 || wps == 16) || wps * 32 > threads)
                return bfail(PJ_EINVAL, "pj_batch_create: item " + std::to_string(i) + ": warps per state");
            sc = pj::make_scratch(m->dev, jac, wps);
            const int sconst = pj::shared_const_doubles(m->N);
            int gmax = threads / (32 * wps);
            if (wps > 1) gmax = std::min(gmax, 15);
            while (gmax > 0 && (size_t(sconst) + size_t(sc.total) * gmax) * 8 > budget) --gmax;
            groups = is->states_per_cta > 0 ? std::min(is->states_per_cta, gmax) : gmax;
            if (groups < 1)
                return bfail(PJ_EUNSUPPORTED, "pj_batch_create: item " + std::to_string(i) +
                                                  ": one state's working set does not fit in shared memory");
        } else if (!pj::batch_group_shape(*m, jac, threads, budget, &wps, &groups, &sc)) {
            return bfail(PJ_EUNSUPPORTED, "pj_batch_create: item " + std::to_string(i) +
                                              ": one state's working set does not fit in shared memory");
        } else if (is && is->states_per_cta > 0) {
            groups = std::min(groups, is->states_per_cta);
        }
        const int sconst = pj::shared_const_doubles(m->N);
        smem = std::max(smem, (size_t(sconst) + size_t(sc.total) * groups) * 8);
        pj::BatchItem &b = bi[i];
        b.m = m->dev_model;
        b.sc = sc;
        b.io = pj::BatchIO{it.T, it.P, it.Y, it.ldy, it.jac, it.ldj, it.dydt, it.ldd};
        b.wps = wps;
        b.groups = groups;
        b.shared_const = sconst;
        cost[i] = double(m->R) * 60.0 + double(m->N + 1) * (m->N + 1);   // rough per-state work
    }
    // tiles: consecutive states of one item, costliest first; by default four rounds of the item's
    // groups, but at most pj::kTileWork of work (whole rounds), so that the launch does not end on
    // one CTA finishing a long tile of a costly model
    std::vector<pj::BatchTile> tiles;
    for (int i = 0; i < n_items; ++i) {
        const long long g = bi[i].groups;
        const long long by_work = std::max<long long>(g, (long long)(pj::kTileWork / cost[i]) / g * g);
        const long long ts = (item_shapes && item_shapes[i].tile_states > 0) ? item_shapes[i].tile_states
                             : tile_req > 0 ? tile_req : std::min(4LL * g, by_work);
        for (long long b = 0; b < items[i].n; b += ts) {
            pj::BatchTile t{};
            t.item = i;
            t.begin = b;
            t.count = std::min<long long>(ts, items[i].n - b);
            tiles.push_back(t);
        }
    }
    std::stable_sort(tiles.begin(), tiles.end(), [&](const pj::BatchTile &a, const pj::BatchTile &b) {
        return cost[a.item] * a.count > cost[b.item] * b.count;
    });
    pj_batch *bt = new (std::nothrow) pj_batch();
    if (!bt) return bfail(PJ_ENOMEM, "host allocation failed");
    for (int i = 0; i < n_items; ++i) {               // slot of each item: its (model, group width)
        int slot = -1;
        for (size_t k = 0; k < bt->slot_mech.size(); ++k)
            if (bt->slot_mech[k] == items[i].mech && bt->slot_wps[k] == bi[i].wps) slot = int(k);
        if (slot < 0) {
            slot = int(bt->slot_mech.size());
            bt->slot_mech.push_back(items[i].mech);
            bt->slot_wps.push_back(bi[i].wps);
        }
        bi[i].pad = slot;
    }
    bt->items = bi;
    bt->tiles = tiles;
    for (int i = 0; i < n_items; ++i)
        bt->auto_width.push_back(!(item_shapes && item_shapes[i].warps_per_state > 0));
    bt->which = which;
    bt->device = dev;
    bt->threads = threads;
    bt->ctas_per_sm = ctas;
    bt->sms = sms;
    bt->smem = smem;
    bt->ntiles = int(tiles.size());
    const size_t o_items = 0, o_tiles = (sizeof(pj::BatchItem) * n_items + 255) & ~size_t(255);
    const size_t o_ctr = (o_tiles + sizeof(pj::BatchTile) * std::max<size_t>(1, tiles.size()) + 255) & ~size_t(255);
    const size_t bytes = o_ctr + sizeof(int) * pj::kBatchSpecMaxSlots;
    if ((e = cudaMalloc(&bt->dev, bytes)) != cudaSuccess) {
        delete bt;
        cudaGetLastError();
        return bfail(PJ_ENOMEM, std::string("batch plan device memory: ") + cudaGetErrorString(e));
    }
    char *d = static_cast<char *>(bt->dev);
    if ((e = cudaMemcpy(d + o_items, bi.data(), sizeof(pj::BatchItem) * n_items, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (!tiles.empty() &&
         (e = cudaMemcpy(d + o_tiles, tiles.data(), sizeof(pj::BatchTile) * tiles.size(), cudaMemcpyHostToDevice)) !=
             cudaSuccess) ||
        (e = pj::prepare_batch_kernel(jac, smem, nullptr)) != cudaSuccess) {
        cudaFree(bt->dev);
        delete bt;
        return bcuda(e, "batch plan upload");
    }
    bt->params.items = reinterpret_cast<const pj::BatchItem *>(d + o_items);
    bt->params.tiles = reinterpret_cast<const pj::BatchTile *>(d + o_tiles);
    bt->params.ntiles = bt->ntiles;
    bt->params.counter = reinterpret_cast<int *>(d + o_ctr);
    *out = bt;
    return PJ_OK;
}

int pj_batch_run(pj_batch *b, void *stream) {
    if (!b) return bfail(PJ_EINVAL, "pj_batch_run: null plan");
    if (b->ntiles == 0) return PJ_OK;
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return bcuda(e, "cudaGetDevice");
    if (cur != b->device) return bfail(PJ_EINVAL, "pj_batch_run: the current device is not the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int counters = b->spec ? b->spec->slots : 1;  // the specialised kernel: one per slot
    if ((e = cudaMemsetAsync(b->params.counter, 0, sizeof(int) * counters, st)) != cudaSuccess)
        return bcuda(e, "counter reset");
    const int blocks = std::max(1, std::min(b->sms * b->ctas_per_sm, b->ntiles));
    if (b->spec) {                                    // the kernel specialised for this plan
        const void *k = reinterpret_cast<const void *>(b->spec->kern);
        pj::BatchParams p = b->params;
        p.items = b->spec->items;
        p.tiles = b->spec->tiles;
        void *args[] = {&p};
        e = cudaLaunchKernel(k, dim3(blocks), dim3(b->threads), args, b->spec->smem, st);
    } else {
        // the kernel's dynamic shared memory limit is one per process: another plan may have set
        // a smaller one since this plan was built
        if ((e = pj::prepare_batch_kernel(b->which == 0, b->smem, nullptr)) != cudaSuccess)
            return bcuda(e, "batch kernel attribute");
        e = pj::launch_batch(b->params, b->which == 0, blocks, b->threads, b->smem, st);
    }
    if (e != cudaSuccess) return bcuda(e, "batch kernel launch");
    return PJ_OK;
}

int pj_batch_info(const pj_batch *b, int *n_tiles, size_t *smem_bytes, int *threads_per_cta) {
    if (!b) return bfail(PJ_EINVAL, "pj_batch_info: null plan");
    if (n_tiles) *n_tiles = b->ntiles;
    if (smem_bytes) *smem_bytes = b->smem;
    if (threads_per_cta) *threads_per_cta = b->threads;
    return PJ_OK;
}

int pj_batch_specialize(pj_batch *b, int enable) {
    if (!b) return bfail(PJ_EINVAL, "pj_batch_specialize: null plan");
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return bcuda(e, "cudaGetDevice");
    if (cur != b->device) return bfail(PJ_EINVAL, "pj_batch_specialize: the current device is not the plan's device");
    if (!enable) {
        pj::batch_spec_release(b);
        return PJ_OK;
    }
    std::string err;
    const int rc = pj::specialize_batch(b, &err);
    if (rc != PJ_OK) return bfail(rc, "pj_batch_specialize: " + err);
    return PJ_OK;
}

int pj_batch_spec_info(const pj_batch *b, int *active, int *slots, double *compile_seconds, size_t *cubin_bytes) {
    if (!b) return bfail(PJ_EINVAL, "pj_batch_spec_info: null plan");
    if (active) *active = b->spec != nullptr;
    if (slots) *slots = b->spec ? b->spec->slots : int(b->slot_mech.size());
    if (compile_seconds) *compile_seconds = b->spec ? b->spec->compile_seconds : 0.0;
    if (cubin_bytes) *cubin_bytes = b->spec ? b->spec->cubin_bytes : 0;
    return PJ_OK;
}

void pj_batch_free(pj_batch *b) {
    if (!b) return;
    pj::batch_spec_release(b);
    if (b->dev) cudaFree(b->dev);
    delete b;
}

}  // extern "C"
