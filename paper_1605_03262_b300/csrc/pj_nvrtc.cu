// Per-model specialised evaluation kernels, compiled at run time with NVRTC: the paper's
// code-generation approach (per-mechanism source, compiled for the mechanism) applied to this
// library's kernels. The device code is the library's own (pj_device_kernels.cuh, embedded at
// build time); what is specialised is every model size and shared-memory offset the data-driven
// kernel reads from its parameter block (species, reactions, b-slots, schedule and chunk counts,
// scratch layout, states per CTA), which become compile-time constants, so that index arithmetic
// and loop bounds fold. The arithmetic and its order are unchanged: a specialised kernel returns the
// same bits as the data-driven one.
//
// NVRTC is loaded on first use (dlopen), so the library itself does not depend on it.
#include <dlfcn.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include <nvrtc.h>

#include "../../include/pyjac_b300.h"
#include "pj_internal.h"

namespace pj {
namespace {

#include "pj_embedded_src.inc"   // kSrcFastmath, kSrcDevice, kSrcDeviceKernels (written by build.py)

struct NvrtcApi {
    bool ok = false;
    std::string why;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

const NvrtcApi &nvrtc_api() {
    static NvrtcApi api;
    static std::once_flag once;
    std::call_once(once, [] {
        void *h = nullptr;
        for (const char *name : {"libnvrtc.so.13", "libnvrtc.so"})
            if ((h = dlopen(name, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!h) {
            api.why = "NVRTC (libnvrtc.so.13) could not be loaded";
            return;
        }
        api.create = reinterpret_cast<decltype(api.create)>(dlsym(h, "nvrtcCreateProgram"));
        api.compile = reinterpret_cast<decltype(api.compile)>(dlsym(h, "nvrtcCompileProgram"));
        api.log_size = reinterpret_cast<decltype(api.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        api.log = reinterpret_cast<decltype(api.log)>(dlsym(h, "nvrtcGetProgramLog"));
        api.cubin_size = reinterpret_cast<decltype(api.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        api.cubin = reinterpret_cast<decltype(api.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        api.ok = api.create && api.compile && api.log_size && api.log && api.cubin_size && api.cubin && api.destroy;
        if (!api.ok) api.why = "NVRTC lacks an expected entry point";
    });
    return api;
}

// Exact text of a double (hexadecimal floating literal).
std::string hex_double(double v) {
    char b[64];
    std::snprintf(b, sizeof b, "%a", v);
    return b;
}

void emit_model(std::string &s, const DevModel &d) {
    s += "__device__ __forceinline__ void spec_model(pj::DevModel &m) {\n";
    auto f = [&](const char *name, long long v) { s += "    m." + std::string(name) + " = " + std::to_string(v) + ";\n"; };
    f("N", d.N), f("R", d.R), f("nslot", d.nslot), f("nnz", d.nnz), f("ncontrib", d.ncontrib);
    f("ncolent", d.ncolent), f("rpc", d.rpc), f("n_row_chunks", d.n_row_chunks), f("ng", d.ng), f("nh", d.nh);
    f("ncc", d.ncc), f("ngp", d.ngp), f("nhp", d.nhp), f("ncp", d.ncp), f("s_npart", d.s_npart);
    s += "    m.lnPatmR = " + hex_double(d.lnPatmR) + ";\n}\n";
}

void emit_scratch(std::string &s, const char *fn, const Scratch &c) {
    s += "__device__ __forceinline__ void " + std::string(fn) + "(pj::Scratch &c) {\n";
    auto f = [&](const char *name, int v) { s += "    c." + std::string(name) + " = " + std::to_string(v) + ";\n"; };
    f("C", c.C), f("B", c.B), f("dB", c.dB), f("H", c.H), f("cpk", c.cpk), f("Jk0", c.Jk0), f("A", c.A);
    f("Ck", c.Ck), f("f", c.f), f("HS", c.HS), f("red", c.red), f("scal", c.scal), f("q", c.q), f("th", c.th);
    f("a", c.a), f("dH", c.dH), f("b", c.b), f("rows", c.rows), f("part", c.part), f("total", c.total);
    f("rows_per_chunk", c.rows_per_chunk);
    s += "}\n";
}

// Kernel names: index = jac * 2 + cv; 4 = the molar-concentration basis Jacobian.
const char *const kSpecNames[kSpecKernels] = {"pj_spec_dydt_cp", "pj_spec_dydt_cv", "pj_spec_jac_cp",
                                              "pj_spec_jac_cv", "pj_spec_jac_conc"};

std::string spec_source(const pj_mech &m, const LaunchCfg &cj, const LaunchCfg &cd) {
    std::string s = "#include \"pj_device_kernels.cuh\"\nnamespace {\n";
    emit_model(s, m.dev);
    emit_scratch(s, "spec_scratch_jac", make_scratch(m.dev, true, cj.wps));
    emit_scratch(s, "spec_scratch_dydt", make_scratch(m.dev, false, cd.wps));
    s += "}  // namespace\n";
    const int sconst = shared_const_doubles(m.N);
    for (int k = 0; k < kSpecKernels; ++k) {
        const bool jac = k >= 2, cv = k < 4 && (k & 1), conc = k == 4;
        const LaunchCfg &c = jac ? cj : cd;
        // launch bounds of the compiled shape: a CTA of fewer than 512 threads leaves each thread
        // more than 128 registers
        const int threads = c.wps * 32 * c.groups, ctas = c.ctas_per_sm > 0 ? c.ctas_per_sm : 1;
        s += "extern \"C\" __global__ void __launch_bounds__(" + std::to_string(threads) + ", " + std::to_string(ctas) +
             ") " + std::string(kSpecNames[k]) +
             "(const __grid_constant__ pj::KParams p) {\n"
             "    pj::KParams q = p;\n"
             "    spec_model(q.m);\n"
             "    " + std::string(jac ? "spec_scratch_jac" : "spec_scratch_dydt") + "(q.sc);\n"
             "    q.groups = " + std::to_string(c.groups) + ";\n"
             "    q.shared_const = " + std::to_string(sconst) + ";\n"
             "    pj::eval_kernel_body<" + (jac ? "true" : "false") + ", " + std::to_string(c.wps) + ", " +
             (cv ? "true" : "false") + ", " + (conc ? "true" : "false") + ">(q);\n}\n";
    }
    return s;
}


int nvrtc_compile(const NvrtcApi &api, const std::string &src, const char *name, const std::string &arch,
                  std::vector<char> *out, std::string *err);

// Compiles source (with the embedded device headers) for the current device's sm_XXa with NVRTC and
// loads it as a library. PJ_OK, or a status with the reason (the compiler log) in *err.
int compile_and_load(const std::string &src, const char *name, cudaLibrary_t *lib, size_t *cubin_bytes,
                     double *seconds, std::string *err) {
    const NvrtcApi &api = nvrtc_api();
    if (!api.ok) {
        *err = api.why;
        return PJ_EUNSUPPORTED;
    }
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        *err = "no CUDA device";
        return PJ_ECUDA;
    }
    const std::string arch = "-arch=sm_" + std::to_string(prop.major) + std::to_string(prop.minor) + "a";
    const auto t0 = std::chrono::steady_clock::now();
    // compiled code of this process, by target and source: a plan or model specialised again for
    // the same source (another plan over the same models and widths) loads it without compiling
    static std::mutex cache_mu;
    static std::map<std::string, std::vector<char>> cache;
    const std::string key = arch + '\n' + src;
    std::vector<char> bin;
    {
        std::lock_guard<std::mutex> lk(cache_mu);
        auto it = cache.find(key);
        if (it != cache.end()) bin = it->second;
    }
    if (bin.empty()) {
        const int rc = nvrtc_compile(api, src, name, arch, &bin, err);
        if (rc != PJ_OK) return rc;
        std::lock_guard<std::mutex> lk(cache_mu);
        if (cache.size() >= 64) cache.clear();    // bounded: a long-running process keeps at most 64
        cache[key] = bin;
    }
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *cubin_bytes = bin.size();
    cudaError_t e = cudaLibraryLoadData(lib, bin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *lib = nullptr;
        *err = std::string("loading the specialised kernels failed: ") + cudaGetErrorString(e);
        return PJ_ECUDA;
    }
    return PJ_OK;
}

// One NVRTC compilation of src for arch into a cubin.
int nvrtc_compile(const NvrtcApi &api, const std::string &src, const char *name, const std::string &arch,
                  std::vector<char> *out, std::string *err) {
    const char *hdr_src[3] = {kSrcFastmath, kSrcDevice, kSrcDeviceKernels};
    const char *hdr_name[3] = {"pj_fastmath.cuh", "pj_device.h", "pj_device_kernels.cuh"};
    nvrtcProgram prog = nullptr;
    if (api.create(&prog, src.c_str(), name, 3, hdr_src, hdr_name) != NVRTC_SUCCESS) {
        *err = "nvrtcCreateProgram failed";
        return PJ_ECUDA;
    }
    const char *opts[] = {arch.c_str(), "-std=c++17", "-default-device"};
    const nvrtcResult rc = api.compile(prog, 3, opts);
    if (rc != NVRTC_SUCCESS) {
        size_t n = 0;
        api.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) api.log(prog, &log[0]);
        api.destroy(&prog);
        *err = "NVRTC compilation failed: " + log.substr(0, 2000);
        return PJ_ECUDA;
    }
    size_t nbin = 0;
    api.cubin_size(prog, &nbin);
    out->assign(nbin, 0);
    api.cubin(prog, out->data());
    api.destroy(&prog);
    return PJ_OK;
}

// Slots of a batched plan's specialised kernel: the distinct (model, warps per state, states per
// round) triples.
struct SpecSlots {
    std::vector<const pj_mech *> mech;
    std::vector<int> wps, groups;
};

// Source of a batched plan's specialised kernel: per slot a Spec type with the model's sizes and
// scratch layout, then the slots' parts of the persistent loop one after another (run_slot_seq),
// in `order`, each over its range [first[k], first[k + 1]) of the grouped tile table. Launch
// bounds: the plan's CTA size (a CTA of fewer than 512 threads leaves each thread more registers).
std::string batch_spec_source(bool jac, int threads, const SpecSlots &sl, const std::vector<int> &order,
                              const std::vector<int> &first) {
    const char *J = jac ? "true" : "false";
    const int ns = int(sl.mech.size());
    std::string s = "#include \"pj_device_kernels.cuh\"\nextern \"C\" {\n";
    for (int k = 0; k < ns; ++k)   // each slot's DevModel, written by specialize_batch after loading
        s += "__constant__ pj::DevModel pj_slot_model" + std::to_string(k) + ";\n";
    s += "}\nnamespace {\n";
    for (int k = 0; k < ns; ++k) {
        const pj_mech &m = *sl.mech[k];
        std::string body;
        emit_model(body, m.dev);
        emit_scratch(body, "spec_scratch", make_scratch(m.dev, jac, sl.wps[k]));
        // emit_model / emit_scratch write free functions; wrap them as static members of Slot<k>
        std::string wrapped;
        size_t pos = 0;
        while (pos < body.size()) {
            size_t e = body.find('\n', pos);
            std::string line = body.substr(pos, e - pos);
            const std::string pre = "__device__ __forceinline__ void ";
            if (line.compare(0, pre.size(), pre) == 0) line = "    static " + line;
            wrapped += line + "\n";
            pos = e + 1;
        }
        s += "struct Slot" + std::to_string(k) + " {\n" + wrapped +
             "    static constexpr int kGroups = " + std::to_string(sl.groups[k]) +
             ", kSharedConst = " + std::to_string(shared_const_doubles(m.N)) + ";\n"
             "    static __device__ __forceinline__ const pj::DevModel &dev() { return pj_slot_model" +
             std::to_string(k) + "; }\n};\n";
    }
    s += "}  // namespace\n";
    s += "extern \"C\" __global__ void __launch_bounds__(" + std::to_string(threads) +
         ", 1) pj_spec_batch(const __grid_constant__ pj::BatchParams p) {\n";
    for (int x = 0; x < ns; ++x) {
        const int k = order[x];
        s += "    pj::run_slot_seq<" + std::string(J) + ", " + std::to_string(sl.wps[k]) + ", Slot" +
             std::to_string(k) + ">(p, " + std::to_string(k) + ", " + std::to_string(first[x]) + ", " +
             std::to_string(first[x + 1]) + ");\n";
    }
    s += "}\n";
    return s;
}

}  // namespace

// Compiles and loads the specialised kernels of a model for its current launch shapes.
int specialize(pj_mech *m, std::string *err) {
    if (m->jac_cfg.groups < 1 || m->dydt_cfg.groups < 1) {
        *err = "the model's working set does not fit in shared memory";
        return PJ_EUNSUPPORTED;
    }
    const std::string src = spec_source(*m, m->jac_cfg, m->dydt_cfg);
    pj_spec *sp = new pj_spec();
    int rc = compile_and_load(src, "pj_spec.cu", &sp->lib, &sp->cubin_bytes, &sp->compile_seconds, err);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kSpecKernels && rc == PJ_OK && e == cudaSuccess; ++k)
        e = cudaLibraryGetKernel(&sp->kern[k], sp->lib, kSpecNames[k]);
    if (rc == PJ_OK && e != cudaSuccess) {
        cudaGetLastError();
        *err = std::string("loading the specialised kernels failed: ") + cudaGetErrorString(e);
        rc = PJ_ECUDA;
    }
    if (rc != PJ_OK) {
        if (sp->lib) cudaLibraryUnload(sp->lib);
        delete sp;
        return rc;
    }
    sp->jac_cfg = m->jac_cfg;
    sp->dydt_cfg = m->dydt_cfg;
    spec_release(m);
    m->spec = sp;
    return PJ_OK;
}

// Compiles and loads the kernel of a batched plan specialised for its models. Its item table is
// the plan's, except that an item whose group width the data-driven plan chose and had to halve
// gets its model's own width back where the working set fits beside this kernel's smaller static
// shared memory (a width the caller set is kept; at 8 instead of 16 warps per state the
// 360-species model ran 1.45 x the plain kernel's time). Tiles are grouped by slot (slots in decreasing work per state,
// so that the last part has the finest tiles; within a slot, the plan's order). Items and tiles
// are uploaded to device memory of the specialisation's own.
int specialize_batch(pj_batch *b, std::string *err) {
    const bool jac = b->which == 0;
    const int n = int(b->items.size());
    if (n == 0) {
        *err = "the plan has no items";
        return PJ_EINVAL;
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    const size_t budget = size_t(optin) > kSpecBatchStaticSmem ? size_t(optin) - kSpecBatchStaticSmem : 0;
    std::vector<BatchItem> items = b->items;
    SpecSlots sl;
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        BatchItem &it = items[i];
        const pj_mech *m = b->slot_mech[it.pad];
        const int w = (jac ? m->jac_cfg : m->dydt_cfg).wps;
        if (b->auto_width[i] && w > it.wps && w * 32 <= b->threads) {
            const Scratch sc = make_scratch(m->dev, jac, w);
            int gmax = b->threads / (32 * w);
            if (w > 1) gmax = std::min(gmax, 15);
            while (gmax > 0 && (size_t(it.shared_const) + size_t(sc.total) * gmax) * 8 > budget) --gmax;
            if (gmax >= 1) {
                it.wps = w;
                it.sc = sc;
                it.groups = gmax;
            }
        }
        smem = std::max(smem, (size_t(it.shared_const) + size_t(it.sc.total) * it.groups) * 8);
        int slot = -1;
        for (size_t k = 0; k < sl.mech.size(); ++k)
            if (sl.mech[k] == m && sl.wps[k] == it.wps && sl.groups[k] == it.groups) slot = int(k);
        if (slot < 0) {
            slot = int(sl.mech.size());
            sl.mech.push_back(m);
            sl.wps.push_back(it.wps);
            sl.groups.push_back(it.groups);
        }
        it.pad = slot;
    }
    const int ns = int(sl.mech.size());
    if (ns > kBatchSpecMaxSlots) {
        *err = "the plan has more than " + std::to_string(kBatchSpecMaxSlots) + " parts ((model, group width, states per round) triples)";
        return PJ_EUNSUPPORTED;
    }
    std::vector<int> order(ns);
    for (int k = 0; k < ns; ++k) order[k] = k;
    auto work = [&](int k) { const pj_mech &m = *sl.mech[k]; return double(m.R) * 60.0 + double(m.N + 1) * (m.N + 1); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work(a) > work(c); });
    // tiles of costly models are cut to at most kTileWork of work (but whole rounds), so that the
    // persistent loop's end is not one CTA finishing a long tile of the 360-species model
    std::vector<BatchTile> grouped;
    std::vector<int> first(ns + 1, 0);
    for (int x = 0; x < ns; ++x) {
        first[x] = int(grouped.size());
        const long long per = std::max<long long>(1, (long long)(kTileWork / work(order[x])));
        for (const BatchTile &t : b->tiles) {
            if (items[t.item].pad != order[x]) continue;
            const long long g = items[t.item].groups;
            const long long step = std::max(g, per / g * g);
            for (long long a = 0; a < t.count; a += step) {
                BatchTile u = t;
                u.begin = t.begin + a;
                u.count = std::min(step, t.count - a);
                grouped.push_back(u);
            }
        }
    }
    first[ns] = int(grouped.size());
    const std::string src = batch_spec_source(jac, b->threads, sl, order, first);
    pj_batch_spec *sp = new pj_batch_spec();
    int rc = compile_and_load(src, "pj_spec_batch.cu", &sp->lib, &sp->cubin_bytes, &sp->compile_seconds, err);
    cudaError_t e = cudaSuccess;
    if (rc == PJ_OK && (e = cudaLibraryGetKernel(&sp->kern, sp->lib, "pj_spec_batch")) != cudaSuccess) {
        *err = std::string("loading the specialised batch kernel failed: ") + cudaGetErrorString(e);
        rc = PJ_ECUDA;
    }
    for (int k = 0; k < ns && rc == PJ_OK; ++k) {  // the slots' DevModels into constant memory
        void *dptr = nullptr;
        size_t bytes = 0;
        const std::string name = "pj_slot_model" + std::to_string(k);
        e = cudaLibraryGetGlobal(&dptr, &bytes, sp->lib, name.c_str());
        if (e == cudaSuccess && bytes != sizeof(DevModel)) e = cudaErrorInvalidValue;
        if (e == cudaSuccess) e = cudaMemcpy(dptr, &sl.mech[k]->dev, sizeof(DevModel), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            *err = "writing " + name + ": " + cudaGetErrorString(e);
            rc = PJ_ECUDA;
        }
    }
    if (rc == PJ_OK) {                             // the kernel's static shared memory fits beside
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(sp->kern));
        if (e == cudaSuccess && fa.sharedSizeBytes > kSpecBatchStaticSmem) {
            *err = "the specialised batch kernel's static shared memory exceeds its reserve";
            rc = PJ_EUNSUPPORTED;
        } else if (e == cudaSuccess) {
            e = cudaFuncSetAttribute(reinterpret_cast<const void *>(sp->kern),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        }
        if (rc == PJ_OK && e != cudaSuccess) {
            *err = std::string("specialised batch kernel attributes: ") + cudaGetErrorString(e);
            rc = PJ_ECUDA;
        }
    }
    if (rc == PJ_OK) {                             // items | tiles in one device buffer
        const size_t o_tiles = (sizeof(BatchItem) * n + 255) & ~size_t(255);
        const size_t bytes = o_tiles + sizeof(BatchTile) * std::max<size_t>(1, grouped.size());
        e = cudaMalloc(&sp->dev, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(sp->dev, items.data(), sizeof(BatchItem) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !grouped.empty())
            e = cudaMemcpy(static_cast<char *>(sp->dev) + o_tiles, grouped.data(), sizeof(BatchTile) * grouped.size(),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            *err = std::string("the specialised kernel's item and tile tables: ") + cudaGetErrorString(e);
            rc = PJ_ECUDA;
        }
        sp->items = static_cast<BatchItem *>(sp->dev);
        sp->tiles = reinterpret_cast<BatchTile *>(static_cast<char *>(sp->dev) + o_tiles);
    }
    if (rc != PJ_OK) {
        cudaGetLastError();
        if (sp->dev) cudaFree(sp->dev);
        if (sp->lib) cudaLibraryUnload(sp->lib);
        delete sp;
        return rc;
    }
    sp->slots = ns;
    sp->smem = smem;
    batch_spec_release(b);
    b->spec = sp;
    return PJ_OK;
}

void batch_spec_release(pj_batch *b) {
    if (!b->spec) return;
    if (b->spec->dev) cudaFree(b->spec->dev);
    if (b->spec->lib) cudaLibraryUnload(b->spec->lib);
    delete b->spec;
    b->spec = nullptr;
}

void spec_release(pj_mech *m) {
    if (!m->spec) return;
    if (m->spec->lib) cudaLibraryUnload(m->spec->lib);
    delete m->spec;
    m->spec = nullptr;
}

const void *spec_kernel(const pj_mech *m, bool jac, bool cv, const LaunchCfg &c) {
    const pj_spec *sp = m->spec;
    if (!sp) return nullptr;
    const LaunchCfg &sc = jac ? sp->jac_cfg : sp->dydt_cfg;
    if (sc.wps != c.wps || sc.groups != c.groups) return nullptr;
    return reinterpret_cast<const void *>(sp->kern[(jac ? 2 : 0) + (cv ? 1 : 0)]);
}

const void *spec_conc_kernel(const pj_mech *m, const LaunchCfg &c) {
    const pj_spec *sp = m->spec;
    if (!sp || sp->jac_cfg.wps != c.wps || sp->jac_cfg.groups != c.groups) return nullptr;
    return reinterpret_cast<const void *>(sp->kern[4]);
}

}  // namespace pj
