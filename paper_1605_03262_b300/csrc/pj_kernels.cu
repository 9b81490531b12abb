// Host side of the evaluation kernels (device code in pj_device_kernels.cuh): scratch layout,
// launch helpers, and the batched launch without allocation.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/pyjac_b300.h"
#include "pj_internal.h"
#include "pj_device_kernels.cuh"

namespace pj {

// ---------------------------------------------------------------------------------------------
// host-side launch helpers

Scratch make_scratch(const DevModel &m, bool jac, int wps) {
    const int N = m.N, R = m.R;
    Scratch sc{};
    int o = 0;
    auto take = [&](int n) {
        int r = o;
        o += (n + 1) & ~1;   // keep every array 16-byte aligned
        return r;
    };
    sc.C = take(N);
    sc.B = take(N);
    sc.H = take(N);
    sc.cpk = take(N);
    sc.f = take(N);
    sc.red = take(8);
    sc.scal = take(kSNumScalars);
    sc.q = take(R + 1);
    if (jac) {
        sc.dB = take(N);
        sc.Jk0 = take(N);
        sc.A = take(N);
        sc.Ck = take(N);
        sc.HS = take(N);
        sc.th = take(R + 1);
        sc.a = take(R + 1);
        sc.dH = take(R + 1);
        sc.b = take(m.nslot + 1);
        sc.rows_per_chunk = m.rpc;
        // the row-staging buffers and the gather's partial sums are never live at the same time
        sc.rows = take(std::max(wps * row_stride(m), 3 * m.ngp + m.nhp + m.ncp));
        sc.part = sc.rows;
    } else {
        sc.dB = sc.Jk0 = sc.A = sc.Ck = sc.HS = sc.th = sc.a = sc.dH = sc.b = sc.rows = 0;
        sc.rows_per_chunk = 0;
        sc.part = take(m.ngp);
    }
    // The reaction stage reads the same species of several states at once (group g at g * total):
    // a total of 2 mod 16 doubles puts up to eight groups in eight different pairs of shared-memory
    // banks (a total of 0 or 8 mod 16 would put several in one pair and serialise their loads).
    o += (2 - o % 16 + 16) % 16;
    sc.total = o;
    return sc;
}

bool batch_group_shape(const pj_mech &m, bool jac, int threads, size_t budget, int *wps, int *groups, Scratch *sc) {
    const int sconst = shared_const_doubles(m.N);
    int w = (jac ? m.jac_cfg : m.dydt_cfg).wps;
    while (w * 32 > threads && w > 1) w /= 2;
    for (; w >= 1; w /= 2) {   // results do not depend on the width; narrower groups stage fewer rows
        const Scratch s = make_scratch(m.dev, jac, w);
        int g = threads / (32 * w);
        if (w > 1) g = std::min(g, 15);
        while (g > 0 && (size_t(sconst) + size_t(s.total) * g) * 8 > budget) --g;
        if (g >= 1) {
            *wps = w;
            *groups = g;
            *sc = s;
            return true;
        }
    }
    return false;
}

int shared_const_doubles(int N) { return 128 + (((2 * N) + 1) & ~1); }

template <bool JAC, bool CV>
static cudaError_t launch_t(const KParams &p, int wps, int blocks, size_t smem, cudaStream_t stream) {
    const int threads = wps * 32 * p.groups;
    cudaError_t e = cudaSuccess;
#define PJ_CASE(W)                                                                                       \
    case W:                                                                                              \
        e = cudaFuncSetAttribute(pj_eval_kernel<JAC, W, CV>, cudaFuncAttributeMaxDynamicSharedMemorySize,\
                                 int(smem));                                                             \
        if (e != cudaSuccess) return e;                                                                  \
        pj_eval_kernel<JAC, W, CV><<<blocks, threads, smem, stream>>>(p);                               \
        return cudaGetLastError();
    switch (wps) {
        PJ_CASE(1)
        PJ_CASE(2)
        PJ_CASE(4)
        PJ_CASE(8)
        PJ_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef PJ_CASE
}

cudaError_t launch_eval(const KParams &p, bool jac, bool cv, int wps, int blocks, size_t smem, cudaStream_t stream) {
    if (cv) return jac ? launch_t<true, true>(p, wps, blocks, smem, stream) : launch_t<false, true>(p, wps, blocks, smem, stream);
    return jac ? launch_t<true, false>(p, wps, blocks, smem, stream) : launch_t<false, false>(p, wps, blocks, smem, stream);
}

cudaError_t launch_conc(const KParams &p, int wps, int blocks, size_t smem, cudaStream_t stream) {
    const int threads = wps * 32 * p.groups;
    cudaError_t e = cudaSuccess;
#define PJ_CASE(W)                                                                                        \
    case W:                                                                                               \
        e = cudaFuncSetAttribute(pj_eval_kernel<true, W, false, true>,                                    \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));                 \
        if (e != cudaSuccess) return e;                                                                   \
        pj_eval_kernel<true, W, false, true><<<blocks, threads, smem, stream>>>(p);                       \
        return cudaGetLastError();
    switch (wps) {
        PJ_CASE(1)
        PJ_CASE(2)
        PJ_CASE(4)
        PJ_CASE(8)
        PJ_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef PJ_CASE
}

cudaError_t prepare_batch_kernel(bool jac, size_t dyn_smem, size_t *static_smem) {
    cudaFuncAttributes a{};
    cudaError_t e = jac ? cudaFuncGetAttributes(&a, pj_batch_kernel<true>) : cudaFuncGetAttributes(&a, pj_batch_kernel<false>);
    if (e != cudaSuccess) return e;
    if (static_smem) *static_smem = a.sharedSizeBytes;
    if (dyn_smem == 0) return cudaSuccess;
    return jac ? cudaFuncSetAttribute(pj_batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn_smem))
               : cudaFuncSetAttribute(pj_batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn_smem));
}

cudaError_t launch_batch(const BatchParams &p, bool jac, int blocks, int threads, size_t smem, cudaStream_t stream) {
    if (jac) pj_batch_kernel<true><<<blocks, threads, smem, stream>>>(p);
    else pj_batch_kernel<false><<<blocks, threads, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace pj

// ---------------------------------------------------------------------------------------------
// Batched launch without any allocation (pj_batch_run_noalloc).
//
// Some callers cannot allocate device memory in their call path: a solver or CFD code that owns a
// fixed memory pool and forbids cudaMalloc/cudaFree inside its time step (both can synchronise the
// device and fragment the pool), or code that must not meet an allocation failure mid-run. For
// them the batched launch passes its item table and tile bounds to the kernel by value (a kernel
// parameter block, at most 64 items) and keeps its one piece of device scratch, the tile counter
// that the CTAs draw tiles from, in the fixed static device array below instead of a cudaMalloc'd
// plan. The caller still passes the state inputs and the outputs.

namespace pj {

constexpr int kNoAllocMaxItems = 64;   // largest number of items one call accepts (parameter space)

// The launch's table, copied into the kernel's parameter space at launch (about 13 KB of the 32 KB
// that a kernel's parameters may take): nothing of it lives in device memory.
struct NoAllocTable {
    int ntiles, n_items;
    int *counter;                      // tile counter in device memory, zeroed before every launch
    int tile_first[kNoAllocMaxItems + 1];   // first tile of each item; tile_first[n_items] = ntiles
    long long tile_states[kNoAllocMaxItems];
    long long n_states[kNoAllocMaxItems];
    BatchItem items[kNoAllocMaxItems];
};
static_assert(sizeof(NoAllocTable) < 32000, "kernel parameter block");

// Device scratch of one launch: the tile counter, padded to one 256-byte line.
constexpr int kNoAllocScratchInts = 64;
// The array (256 bytes): held by every device that loads the library, until the process exits.
static __device__ __align__(256) int g_noalloc_scratch[kNoAllocScratchInts];

template <bool JAC>
__global__ void __launch_bounds__(512, 1) pj_batch_noalloc_kernel(const __grid_constant__ NoAllocTable p) {
    extern __shared__ __align__(16) double smem[];
    __shared__ int s_tile, s_item;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const int tile = atomicAdd(p.counter, 1);
            int it = 0;
            if (tile < p.ntiles)
                while (it + 1 < p.n_items && tile >= p.tile_first[it + 1]) ++it;   // skips items without tiles
            s_tile = tile;
            s_item = it;
        }
        __syncthreads();
        const int tile = s_tile, item = s_item;
        if (tile >= p.ntiles) break;
        const BatchItem &it = p.items[item];
        const long long ts = p.tile_states[item];
        const long long begin = (long long)(tile - p.tile_first[item]) * ts;
        const long long end = min(begin + ts, p.n_states[item]);
        Grp g;
        g.wps = it.wps;
        g.G = it.wps * 32;
        g.grp = threadIdx.x / g.G;
        g.t = threadIdx.x - g.grp * g.G;
        g.lane = threadIdx.x & 31;
        g.wg = g.t >> 5;
        double *S = smem + it.shared_const + size_t(g.grp) * it.sc.total;
        const DevModel *__restrict__ mp = it.m;       // read in place (see pj_batch_kernel)
        if (item != cur) {
            load_model_consts(*mp, smem);
            if (g.grp < it.groups) init_neutral<JAC>(*mp, it.sc, S, g.t);
            cur = item;
            __syncthreads();
        }
        run_tile<JAC>(*mp, it, smem, begin, end, g);
        __syncthreads();
    }
}

}  // namespace pj

namespace {

// Device address of g_noalloc_scratch, looked up once per device (the symbol's host-side name is
// only a stand-in and must never be handed to a kernel).
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {nullptr};

int noalloc_fail(int code, const std::string &msg) { return pj::set_error(code, msg); }

}  // namespace

namespace {

// Builds the item table of a batched launch on the host, zeroes the tile counter at `counter` (in
// the static array or a caller's workspace) with an asynchronous memset on the stream, and
// launches the persistent batched kernel with the table as its parameter block. Nothing waits on
// the host for earlier work on the stream, and no host memory is read after the call returns.
int batch_run_table(const char *fn, const pj_batch_item *items, int n_items, int which, int tile_states, int dev,
                    int *counter, cudaStream_t st) {
    using namespace pj;
    const std::string f(fn);
    cudaError_t e;
    int sms = 0, optin = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const bool jac = which == 0;
    cudaFuncAttributes fa{};
    e = jac ? cudaFuncGetAttributes(&fa, pj_batch_noalloc_kernel<true>)
            : cudaFuncGetAttributes(&fa, pj_batch_noalloc_kernel<false>);
    if (e != cudaSuccess) return noalloc_fail(PJ_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    const size_t budget = size_t(optin) > fa.sharedSizeBytes ? size_t(optin) - fa.sharedSizeBytes : 0;
    const int threads = 512;

    NoAllocTable h;
    std::memset(&h, 0, sizeof(h));
    h.n_items = n_items;
    h.counter = counter;
    size_t smem = 0;
    int ntiles = 0;
    for (int i = 0; i < n_items; ++i) {
        const pj_batch_item &x = items[i];
        const pj_mech *m = x.mech;
        if (!m || x.n < 0) return noalloc_fail(PJ_EINVAL, f + ": null model or n < 0");
        if (m->device != dev) return noalloc_fail(PJ_EINVAL, f + ": model lives on another device");
        const int64_t N = m->N, nn = (N + 1) * (N + 1);
        if (x.ldy < N || (jac && x.ldj < nn) || ((!jac || x.dydt) && x.ldd < N + 1))
            return noalloc_fail(PJ_EINVAL, f + ": leading dimension too small");
        if (x.n > 0 && (!x.T || !x.P || !x.Y || (jac && !x.jac) || (!jac && !x.dydt)))
            return noalloc_fail(PJ_EINVAL, f + ": null input or output pointer");
        int wps = 0, groups = 0;
        Scratch sc{};
        if (!batch_group_shape(*m, jac, threads, budget, &wps, &groups, &sc))
            return noalloc_fail(PJ_EUNSUPPORTED, f + ": state working set exceeds shared memory");
        const int sconst = shared_const_doubles(m->N);
        smem = std::max(smem, (size_t(sconst) + size_t(sc.total) * groups) * 8);
        BatchItem &b = h.items[i];
        b.m = m->dev_model;
        b.sc = sc;
        b.io = BatchIO{x.T, x.P, x.Y, x.ldy, x.jac, x.ldj, x.dydt, x.ldd};
        b.wps = wps;
        b.groups = groups;
        b.shared_const = sconst;
        const long long ts = tile_states > 0 ? tile_states : 4LL * groups;
        h.tile_states[i] = ts;
        h.n_states[i] = x.n;
        h.tile_first[i] = ntiles;
        const long long nt = (x.n + ts - 1) / ts;
        if (ntiles + nt > 0x7fffffffLL) return noalloc_fail(PJ_EINVAL, f + ": too many tiles");
        ntiles += int(nt);
    }
    h.tile_first[n_items] = ntiles;
    h.ntiles = ntiles;
    if (ntiles == 0) return PJ_OK;
    // what must start at zero: the tile counter. A call still running on the GPU with the same
    // counter would race with this one.
    e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return noalloc_fail(PJ_ECUDA, std::string("counter reset: ") + cudaGetErrorString(e));
    e = jac ? cudaFuncSetAttribute(pj_batch_noalloc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))
            : cudaFuncSetAttribute(pj_batch_noalloc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return noalloc_fail(PJ_ECUDA, std::string("kernel attribute: ") + cudaGetErrorString(e));
    const int blocks = std::max(1, std::min(sms, ntiles));
    if (jac) pj_batch_noalloc_kernel<true><<<blocks, threads, smem, st>>>(h);
    else pj_batch_noalloc_kernel<false><<<blocks, threads, smem, st>>>(h);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(PJ_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return PJ_OK;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int pj_batch_run_noalloc(const pj_batch_item *items, int n_items,
                                                                          int which, int tile_states, void *stream) {
    using namespace pj;
    if (!items || n_items < 1 || (which != 0 && which != 1) || tile_states < 0)
        return noalloc_fail(PJ_EINVAL, "pj_batch_run_noalloc: bad argument");
    if (n_items > kNoAllocMaxItems)
        return noalloc_fail(PJ_EINVAL, "pj_batch_run_noalloc: " + std::to_string(n_items) +
                                           " items, more than one call's parameter table holds (" +
                                           std::to_string(kNoAllocMaxItems) + ")");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(PJ_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return noalloc_fail(PJ_EUNSUPPORTED, "pj_batch_run_noalloc: device index above 63");
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            // first call on this device: the set-up (do it before any stream capture)
            e = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_noalloc_ptr[dev] = nullptr;
                return noalloc_fail(PJ_ECUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                                  cudaGetErrorString(e));
            }
        }
        scratch = g_noalloc_ptr[dev];
    }
    return batch_run_table("pj_batch_run_noalloc", items, n_items, which, tile_states, dev, static_cast<int *>(scratch),
                           static_cast<cudaStream_t>(stream));
}

extern "C" __attribute__((visibility("default"))) size_t pj_batch_workspace_bytes(void) {
    return sizeof(int) * pj::kNoAllocScratchInts;
}

extern "C" __attribute__((visibility("default"))) int pj_batch_run_ws(const pj_batch_item *items, int n_items,
                                                                     int which, int tile_states, void *workspace,
                                                                     size_t workspace_bytes, void *stream) {
    using namespace pj;
    if (!items || n_items < 1 || (which != 0 && which != 1) || tile_states < 0)
        return noalloc_fail(PJ_EINVAL, "pj_batch_run_ws: bad argument");
    if (n_items > kNoAllocMaxItems)
        return noalloc_fail(PJ_EINVAL, "pj_batch_run_ws: " + std::to_string(n_items) + " items, more than a workspace holds (" +
                                           std::to_string(kNoAllocMaxItems) + ")");
    if (!workspace || workspace_bytes < sizeof(int) * kNoAllocScratchInts || (reinterpret_cast<uintptr_t>(workspace) & 15))
        return noalloc_fail(PJ_EINVAL, "pj_batch_run_ws: workspace null, smaller than pj_batch_workspace_bytes() or "
                                       "not 16-byte aligned");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(PJ_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    cudaPointerAttributes pa{};
    e = cudaPointerGetAttributes(&pa, workspace);
    if (e != cudaSuccess || pa.type != cudaMemoryTypeDevice || pa.device != dev) {
        cudaGetLastError();
        return noalloc_fail(PJ_EINVAL, "pj_batch_run_ws: workspace is not device memory of the current device");
    }
    return batch_run_table("pj_batch_run_ws", items, n_items, which, tile_states, dev, static_cast<int *>(workspace),
                           static_cast<cudaStream_t>(stream));
}
