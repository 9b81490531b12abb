// C ABI of libpyjacb300.so: argument checking, model upload and kernel launch (include/pyjac_b300.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <iterator>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/pyjac_b300.h"
#include "pj_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(PJ_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

struct DeviceProps {
    int sms = 0;
    int smem_optin = 0;
};

DeviceProps device_props(int dev) {
    static std::mutex mu;
    static std::vector<DeviceProps> cache;
    std::lock_guard<std::mutex> lk(mu);
    if (int(cache.size()) <= dev) cache.resize(dev + 1);
    if (cache[dev].sms == 0) {
        cudaDeviceGetAttribute(&cache[dev].sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&cache[dev].smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    return cache[dev];
}


size_t smem_bytes(const pj_mech *m, bool jac, const pj::LaunchCfg &c) {
    pj::Scratch sc = pj::make_scratch(m->dev, jac, c.wps);
    return (size_t(pj::shared_const_doubles(m->N)) + size_t(sc.total) * c.groups) * sizeof(double);
}

bool valid_shape(const pj::LaunchCfg &c) {
    const int w = c.wps;
    if (!(w == 1 || w == 2 || w == 4 || w == 8 || w == 16)) return false;
    if (c.groups < 1 || c.ctas_per_sm < 1 || c.ctas_per_sm > 32) return false;
    if (w * 32 * c.groups > 512) return false;
    if (w > 1 && c.groups > 15) return false;   // named barriers 1..15
    return true;
}

// Largest number of states per CTA that fits shared memory, for a given warps-per-state.
pj::LaunchCfg default_cfg(const pj_mech *m, bool jac, int wps) {
    DeviceProps dp = device_props(m->device);
    pj::LaunchCfg c;
    c.wps = wps;
    c.ctas_per_sm = 1;
    int gmax = std::min(wps > 1 ? 15 : 16, 512 / (32 * wps));
    c.groups = 0;
    for (int g = gmax; g >= 1; --g) {
        pj::LaunchCfg t = c;
        t.groups = g;
        if (smem_bytes(m, jac, t) <= size_t(dp.smem_optin)) {
            c.groups = g;
            break;
        }
    }
    return c;
}

pj::LaunchCfg pick_default(const pj_mech *m, bool jac) {
    const int N = m->N;
    int wps = pj::default_wps(N, jac);
    pj::LaunchCfg c = default_cfg(m, jac, wps);
    while (c.groups == 0 && wps < 16) {   // grow the group until one state fits
        wps *= 2;
        c = default_cfg(m, jac, wps);
    }
    return c;
}

bool is_aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

int check_device_ptr(const void *p, int dev, const char *name) {
    if (!p) return fail(PJ_EINVAL, std::string(name) + " is NULL");
    if (!is_aligned8(p)) return fail(PJ_EINVAL, std::string(name) + " is not 8-byte aligned");
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PJ_EINVAL, std::string(name) + " is not a CUDA-accessible pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(PJ_EINVAL, std::string(name) + " is not a device pointer");
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return fail(PJ_EINVAL, std::string(name) + " lives on another device than the model");
    return PJ_OK;
}

template <class T>
size_t push(std::vector<char> &blob, const std::vector<T> &v) {
    size_t off = (blob.size() + 255) & ~size_t(255);
    blob.resize(off + v.size() * sizeof(T) + (v.empty() ? sizeof(T) : 0));
    if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

// P holds pressures (constant-pressure form) or densities (cv: constant-volume form).
int launch(const pj_mech *m, bool jac, bool cv, int64_t n, const double *T, const double *P, const double *Y,
           int64_t ldy, double *jacp, int64_t ldj, double *dydt, int64_t ldd, cudaStream_t stream) {
    const pj::LaunchCfg &c = jac ? m->jac_cfg : m->dydt_cfg;
    if (c.groups < 1)
        return fail(PJ_EUNSUPPORTED, "one state's working set does not fit in shared memory for this model");
    pj::KParams p{};
    p.m = m->dev;
    p.sc = pj::make_scratch(m->dev, jac, c.wps);
    p.n = n;
    p.T = T;
    p.P = P;
    p.Y = Y;
    p.ldy = ldy;
    p.jac = jacp;
    p.ldj = ldj;
    p.dydt = dydt;
    p.ldd = ldd;
    p.groups = c.groups;
    p.shared_const = pj::shared_const_doubles(m->N);
    DeviceProps dp = device_props(m->device);
    long long need = (n + c.groups - 1) / c.groups;
    int blocks = int(std::min<long long>(need, (long long)dp.sms * c.ctas_per_sm));
    size_t smem = smem_bytes(m, jac, c);
    cudaError_t e;
    if (const void *sk = pj::spec_kernel(m, jac, cv, c)) {      // the model's specialised kernel
        e = cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        void *args[] = {&p};
        if (e == cudaSuccess) e = cudaLaunchKernel(sk, dim3(blocks), dim3(c.wps * 32 * c.groups), args, smem, stream);
    } else {
        e = pj::launch_eval(p, jac, cv, c.wps, blocks, smem, stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return PJ_OK;
}

int check_model_device(const pj_mech *m) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (cur != m->device) return fail(PJ_EINVAL, "the current CUDA device is not the model's device");
    return PJ_OK;
}

}  // namespace

int pj::set_error(int code, const std::string &msg) { return fail(code, msg); }

extern "C" {

int pj_version(void) { return 10000; }

const char *pj_last_error(void) { return g_err.c_str(); }

int pj_mech_load(const void *buf, size_t len, pj_mech **out) {
    if (!buf || !out) return fail(PJ_EINVAL, "pj_mech_load: null argument");
    *out = nullptr;
    pj::HostImage im;
    try {
        im = pj::build_image(buf, len);
    } catch (const pj::FormatError &ex) {
        return fail(PJ_EFORMAT, std::string("model format: ") + ex.what());
    } catch (const pj::Unsupported &ex) {
        return fail(PJ_EUNSUPPORTED, std::string("unsupported model: ") + ex.what());
    } catch (const std::bad_alloc &) {
        return fail(PJ_ENOMEM, "host allocation failed while building the model image");
    }
    std::vector<char> blob;
    size_t o_rx = push(blob, im.rx), o_par = push(blob, im.par), o_effsp = push(blob, im.eff_sp),
           o_effeps = push(blob, im.eff_eps), o_sinfo = push(blob, im.slot_info), o_seps = push(blob, im.slot_eps),
           o_th = push(blob, im.thermo), o_tmid = push(blob, im.Tmid), o_W = push(blob, im.W),
           o_iW = push(blob, im.invW), o_D = push(blob, im.Delta), o_spp = push(blob, im.sp_ptr),
           o_spr = push(blob, im.sp_rxn), o_spn = push(blob, im.sp_nu), o_cp = push(blob, im.col_ptr),
           o_cs = push(blob, im.col_slot), o_cr = push(blob, im.col_rxn), o_rp = push(blob, im.row_ptr),
           o_nc = push(blob, im.nnz_col), o_ncp = push(blob, im.nnz_cptr), o_nw = push(blob, im.nnz_wr),
           o_cns = push(blob, im.con_slot), o_cnn = push(blob, im.con_nu), o_cN = push(blob, im.colN_nnz);
    size_t o_gr = push(blob, im.g_rec), o_hr = push(blob, im.h_rec), o_cr2 = push(blob, im.c_rec),
           o_sr = push(blob, im.s_rec), o_sc = push(blob, im.s_chunk), o_gc = push(blob, im.g_chunk),
           o_hc = push(blob, im.h_chunk), o_cc = push(blob, im.c_chunk), o_scc = push(blob, im.s_comb_chunk),
           o_scb = push(blob, im.s_comb), o_gpf = push(blob, im.g_pfirst), o_hpf = push(blob, im.h_pfirst),
           o_cpf = push(blob, im.c_pfirst);
    size_t o_ccp = push(blob, im.cc_ptr), o_ccw = push(blob, im.cc_wr), o_ccc = push(blob, im.cc_col),
           o_dnu = push(blob, im.rx_dnu);
    pj::MathTables tables;
    pj::build_math_tables(tables);
    std::vector<pj::MathTables> tvec(1, tables);
    size_t o_mt = push(blob, tvec);
    std::vector<pj::DevModel> dm_placeholder(1);
    size_t o_dm = push(blob, dm_placeholder);
    pj_mech *m = new (std::nothrow) pj_mech();
    if (!m) return fail(PJ_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&m->device);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "cudaGetDevice");
    }
    e = cudaMalloc(&m->dev_blob, blob.size());
    if (e != cudaSuccess) {
        delete m;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? PJ_ENOMEM : PJ_ECUDA,
                    std::string("cudaMalloc of the model image: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(m->dev_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->dev_blob);
        delete m;
        return cuda_fail(e, "cudaMemcpy of the model image");
    }
    char *b = static_cast<char *>(m->dev_blob);
    pj::DevModel &d = m->dev;
    d.N = im.N;
    d.R = im.R;
    d.nslot = int(im.slot_info.size());
    d.nnz = int(im.nnz_col.size());
    d.ncontrib = int(im.con_slot.size());
    d.ncolent = int(im.col_slot.size());
    d.rx = reinterpret_cast<const pj::RxnDev *>(b + o_rx);
    d.par = reinterpret_cast<const double *>(b + o_par);
    d.eff_sp = reinterpret_cast<const int *>(b + o_effsp);
    d.eff_eps = reinterpret_cast<const double *>(b + o_effeps);
    d.slot_info = reinterpret_cast<const int *>(b + o_sinfo);
    d.slot_eps = reinterpret_cast<const double *>(b + o_seps);
    d.thermo = reinterpret_cast<const double *>(b + o_th);
    d.Tmid = reinterpret_cast<const double *>(b + o_tmid);
    d.W = reinterpret_cast<const double *>(b + o_W);
    d.invW = reinterpret_cast<const double *>(b + o_iW);
    d.Delta = reinterpret_cast<const double *>(b + o_D);
    d.sp_ptr = reinterpret_cast<const int *>(b + o_spp);
    d.sp_rxn = reinterpret_cast<const int *>(b + o_spr);
    d.sp_nu = reinterpret_cast<const double *>(b + o_spn);
    d.col_ptr = reinterpret_cast<const int *>(b + o_cp);
    d.col_slot = reinterpret_cast<const int *>(b + o_cs);
    d.col_rxn = reinterpret_cast<const int *>(b + o_cr);
    d.row_ptr = reinterpret_cast<const int *>(b + o_rp);
    d.nnz_col = reinterpret_cast<const int *>(b + o_nc);
    d.nnz_cptr = reinterpret_cast<const int *>(b + o_ncp);
    d.nnz_wr = reinterpret_cast<const double *>(b + o_nw);
    d.con_slot = reinterpret_cast<const int *>(b + o_cns);
    d.con_nu = reinterpret_cast<const double *>(b + o_cnn);
    d.colN_nnz = reinterpret_cast<const int *>(b + o_cN);
    d.lnPatmR = std::log(pj::kPatm / pj::kR);
    d.rpc = im.rpc;
    d.n_row_chunks = im.n_row_chunks;
    d.ng = im.ng;
    d.nh = im.nh;
    d.ncc = im.ncc;
    d.ngp = im.ngp;
    d.nhp = im.nhp;
    d.ncp = im.ncp;
    d.c_pfirst = reinterpret_cast<const int *>(b + o_cpf);
    d.g_pfirst = reinterpret_cast<const int *>(b + o_gpf);
    d.h_pfirst = reinterpret_cast<const int *>(b + o_hpf);
    d.g_rec = reinterpret_cast<const uint2 *>(b + o_gr);
    d.h_rec = reinterpret_cast<const uint4 *>(b + o_hr);
    d.c_rec = reinterpret_cast<const uint4 *>(b + o_cr2);
    d.s_rec = reinterpret_cast<const uint4 *>(b + o_sr);
    d.s_chunk = reinterpret_cast<const int2 *>(b + o_sc);
    d.g_chunk = reinterpret_cast<const int2 *>(b + o_gc);
    d.h_chunk = reinterpret_cast<const int2 *>(b + o_hc);
    d.c_chunk = reinterpret_cast<const int2 *>(b + o_cc);
    d.s_npart = im.s_npart;
    d.s_comb_chunk = reinterpret_cast<const int2 *>(b + o_scc);
    d.s_comb = reinterpret_cast<const int2 *>(b + o_scb);
    d.tables = reinterpret_cast<const pj::MathTables *>(b + o_mt);
    d.cc_nnz = int(im.cc_col.size());
    d.cc_ptr = reinterpret_cast<const int *>(b + o_ccp);
    d.cc_wr = reinterpret_cast<const double *>(b + o_ccw);
    d.cc_col = reinterpret_cast<const int *>(b + o_ccc);
    d.rx_dnu = reinterpret_cast<const double *>(b + o_dnu);
    d.image = b;
    d.image_bytes = (long long)(blob.size() & ~size_t(15));
    m->dev_model = reinterpret_cast<const pj::DevModel *>(b + o_dm);
    e = cudaMemcpy(b + o_dm, &d, sizeof(d), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->dev_blob);
        delete m;
        return cuda_fail(e, "cudaMemcpy of the model descriptor");
    }
    m->N = im.N;
    m->R = im.R;
    m->NE = im.NE;
    m->dev_bytes = blob.size();
    m->perm = im.perm;
    m->cc_ptr = im.cc_ptr;
    m->cc_col = im.cc_col;
    m->jac_cfg = pick_default(m, true);
    m->dydt_cfg = pick_default(m, false);
    *out = m;
    return PJ_OK;
}

int pj_mech_load_file(const char *path, pj_mech **out) {
    if (!path || !out) return fail(PJ_EINVAL, "pj_mech_load_file: null argument");
    std::ifstream f(path, std::ios::binary);
    if (!f) return fail(PJ_EINVAL, std::string("cannot open ") + path);
    std::vector<char> buf((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
    return pj_mech_load(buf.data(), buf.size(), out);
}

void pj_mech_free(pj_mech *m) {
    if (!m) return;
    if (m->dev_blob) cudaFree(m->dev_blob);
    pj_host_staging_release(m);
    pj::spec_release(m);
    delete m;
}

int pj_mech_info(const pj_mech *m, int *n_species, int *n_reactions, size_t *dev_bytes) {
    if (!m) return fail(PJ_EINVAL, "pj_mech_info: null model");
    if (n_species) *n_species = m->N;
    if (n_reactions) *n_reactions = m->R;
    if (dev_bytes) *dev_bytes = m->dev_bytes;
    return PJ_OK;
}

static int eval_dydt(const char *fn, bool cv, const pj_mech *m, int64_t n, const double *T, const double *P,
                     const double *Y, int64_t ldy, double *dydt, int64_t ldd, void *stream) {
    const std::string f(fn);
    const char *pn = cv ? "rho" : "P";
    if (!m) return fail(PJ_EINVAL, f + ": null model");
    if (n < 0) return fail(PJ_EINVAL, f + ": n < 0");
    if (ldy < m->N) return fail(PJ_EINVAL, f + ": ldy < number of species");
    if (ldd < m->N + 1) return fail(PJ_EINVAL, f + ": ldd < number of species + 1");
    if (n == 0) return PJ_OK;
    int rc;
    if ((rc = check_model_device(m)) || (rc = check_device_ptr(T, m->device, "T")) ||
        (rc = check_device_ptr(P, m->device, pn)) || (rc = check_device_ptr(Y, m->device, "Y")) ||
        (rc = check_device_ptr(dydt, m->device, "dydt")))
        return rc;
    return launch(m, false, cv, n, T, P, Y, ldy, nullptr, 0, dydt, ldd, static_cast<cudaStream_t>(stream));
}

int pj_eval_dydt(const pj_mech *m, int64_t n, const double *T, const double *P, const double *Y, int64_t ldy,
                 double *dydt, int64_t ldd, void *stream) {
    return eval_dydt("pj_eval_dydt", false, m, n, T, P, Y, ldy, dydt, ldd, stream);
}

int pj_eval_dydt_cv(const pj_mech *m, int64_t n, const double *T, const double *rho, const double *Y, int64_t ldy,
                    double *dydt, int64_t ldd, void *stream) {
    return eval_dydt("pj_eval_dydt_cv", true, m, n, T, rho, Y, ldy, dydt, ldd, stream);
}

// Doubles of forward-difference workspace per state: the N perturbed states (T, P, Y[N]), their
// source terms (N x (N+1)) and the state's own source terms (N+1).
static size_t fd_doubles_per_state(int N) { return size_t(N) * (N + 2) + size_t(N) * (N + 1) + size_t(N + 1); }

int pj_fd_workspace_bytes(const pj_mech *m, int64_t n, size_t *bytes) {
    if (!m || n < 0 || !bytes) return fail(PJ_EINVAL, "pj_fd_workspace_bytes: bad argument");
    *bytes = size_t(n) * fd_doubles_per_state(m->N) * sizeof(double);
    return PJ_OK;
}

int pj_eval_jacobian_fd(const pj_mech *m, int64_t n, const double *T, const double *P, const double *Y,
                        int64_t ldy, double *jac, int64_t ldj, void *workspace, size_t workspace_bytes,
                        void *stream) {
    if (!m) return fail(PJ_EINVAL, "pj_eval_jacobian_fd: null model");
    if (n < 0) return fail(PJ_EINVAL, "pj_eval_jacobian_fd: n < 0");
    if (ldy < m->N) return fail(PJ_EINVAL, "pj_eval_jacobian_fd: ldy < number of species");
    const int N = m->N;
    if (ldj < int64_t(N + 1) * (N + 1)) return fail(PJ_EINVAL, "pj_eval_jacobian_fd: ldj < (number of species + 1)^2");
    if (n == 0) return PJ_OK;
    const size_t per = fd_doubles_per_state(N);
    const int64_t chunk = int64_t(std::min<size_t>(size_t(n), workspace_bytes / (per * sizeof(double))));
    if (chunk < 1) return fail(PJ_EINVAL, "pj_eval_jacobian_fd: workspace smaller than one state needs");
    if (reinterpret_cast<uintptr_t>(workspace) & 7) return fail(PJ_EINVAL, "pj_eval_jacobian_fd: workspace not 8-byte aligned");
    int rc;
    if ((rc = check_model_device(m)) || (rc = check_device_ptr(T, m->device, "T")) ||
        (rc = check_device_ptr(P, m->device, "P")) || (rc = check_device_ptr(Y, m->device, "Y")) ||
        (rc = check_device_ptr(jac, m->device, "jac")) || (rc = check_device_ptr(workspace, m->device, "workspace")))
        return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int64_t s0 = 0; s0 < n; s0 += chunk) {
        const int64_t cs = std::min(chunk, n - s0);
        double *Tp = static_cast<double *>(workspace), *Pp = Tp + cs * N, *Yp = Pp + cs * N;
        double *Fp = Yp + cs * N * N, *F0 = Fp + cs * N * (N + 1);
        const double *Ts = T + s0, *Ps = P + s0, *Ys = Y + s0 * ldy;
        if ((rc = launch(m, false, false, cs, Ts, Ps, Ys, ldy, nullptr, 0, F0, N + 1, st))) return rc;
        cudaError_t e = pj::launch_fd_perturb(N, cs, Ts, Ps, Ys, ldy, Tp, Pp, Yp, st);
        if (e != cudaSuccess) return cuda_fail(e, "finite-difference perturbation kernel");
        if ((rc = launch(m, false, false, cs * N, Tp, Pp, Yp, N, nullptr, 0, Fp, N + 1, st))) return rc;
        e = pj::launch_fd_difference(N, cs, Ts, Ys, ldy, F0, Fp, jac + s0 * ldj, ldj, st);
        if (e != cudaSuccess) return cuda_fail(e, "finite-difference column kernel");
    }
    return PJ_OK;
}

static int eval_jacobian(const char *fn, bool cv, const pj_mech *m, int64_t n, const double *T, const double *P,
                         const double *Y, int64_t ldy, double *jac, int64_t ldj, double *dydt, int64_t ldd,
                         void *stream) {
    const std::string f(fn);
    const char *pn = cv ? "rho" : "P";
    if (!m) return fail(PJ_EINVAL, f + ": null model");
    if (n < 0) return fail(PJ_EINVAL, f + ": n < 0");
    if (ldy < m->N) return fail(PJ_EINVAL, f + ": ldy < number of species");
    const int64_t nn = int64_t(m->N + 1) * (m->N + 1);
    if (ldj < nn) return fail(PJ_EINVAL, f + ": ldj < (number of species + 1)^2");
    if (dydt && ldd < m->N + 1) return fail(PJ_EINVAL, f + ": ldd < number of species + 1");
    if (n == 0) return PJ_OK;
    int rc;
    if ((rc = check_model_device(m)) || (rc = check_device_ptr(T, m->device, "T")) ||
        (rc = check_device_ptr(P, m->device, pn)) || (rc = check_device_ptr(Y, m->device, "Y")) ||
        (rc = check_device_ptr(jac, m->device, "jac")))
        return rc;
    if (dydt && (rc = check_device_ptr(dydt, m->device, "dydt"))) return rc;
    return launch(m, true, cv, n, T, P, Y, ldy, jac, ldj, dydt, ldd, static_cast<cudaStream_t>(stream));
}

int pj_eval_jacobian(const pj_mech *m, int64_t n, const double *T, const double *P, const double *Y,
                     int64_t ldy, double *jac, int64_t ldj, double *dydt, int64_t ldd, void *stream) {
    return eval_jacobian("pj_eval_jacobian", false, m, n, T, P, Y, ldy, jac, ldj, dydt, ldd, stream);
}

int pj_eval_jacobian_cv(const pj_mech *m, int64_t n, const double *T, const double *rho, const double *Y,
                        int64_t ldy, double *jac, int64_t ldj, double *dydt, int64_t ldd, void *stream) {
    return eval_jacobian("pj_eval_jacobian_cv", true, m, n, T, rho, Y, ldy, jac, ldj, dydt, ldd, stream);
}

int pj_conc_pattern(const pj_mech *m, int64_t *nnz, int32_t *row_ptr, int32_t *col_idx) {
    if (!m || !nnz) return fail(PJ_EINVAL, "pj_conc_pattern: null argument");
    const int N = m->N;
    const int64_t cc = m->cc_ptr.empty() ? 0 : m->cc_ptr.back();
    *nnz = 2 * int64_t(N + 1) + 2 * int64_t(N - 1) + cc;
    if (!row_ptr && !col_idx) return PJ_OK;
    if (!row_ptr || !col_idx) return fail(PJ_EINVAL, "pj_conc_pattern: give both row_ptr and col_idx, or neither");
    int64_t o = 0;
    for (int r = 0; r < 2; ++r) {                   // T and V rows: dense
        row_ptr[r] = int32_t(o);
        for (int c = 0; c <= N; ++c) col_idx[o++] = c;
    }
    for (int k = 0; k < N - 1; ++k) {               // species rows: T, V, then the pattern
        row_ptr[2 + k] = int32_t(o);
        col_idx[o++] = 0;
        col_idx[o++] = 1;
        for (int e = m->cc_ptr[k]; e < m->cc_ptr[k + 1]; ++e) col_idx[o++] = 2 + m->cc_col[e];
    }
    row_ptr[N + 1] = int32_t(o);
    return PJ_OK;
}

int pj_eval_jacobian_conc(const pj_mech *m, int64_t n, const double *T, const double *P, const double *V,
                          const double *nmol, int64_t ldn, double *jac, int64_t ldj, double *dydt, int64_t ldd,
                          void *stream) {
    const std::string f("pj_eval_jacobian_conc");
    if (!m) return fail(PJ_EINVAL, f + ": null model");
    if (n < 0) return fail(PJ_EINVAL, f + ": n < 0");
    if (m->N < 2) return fail(PJ_EUNSUPPORTED, f + ": the basis needs at least two species");
    if (ldn < m->N - 1) return fail(PJ_EINVAL, f + ": ldn < number of species - 1");
    int64_t nnz = 0;
    pj_conc_pattern(m, &nnz, nullptr, nullptr);
    if (ldj < nnz) return fail(PJ_EINVAL, f + ": ldj < the pattern's number of entries (pj_conc_pattern)");
    if (dydt && ldd < m->N + 1) return fail(PJ_EINVAL, f + ": ldd < number of species + 1");
    if (n == 0) return PJ_OK;
    int rc;
    if ((rc = check_model_device(m)) || (rc = check_device_ptr(T, m->device, "T")) ||
        (rc = check_device_ptr(P, m->device, "P")) || (rc = check_device_ptr(V, m->device, "V")) ||
        (rc = check_device_ptr(nmol, m->device, "nmol")) || (rc = check_device_ptr(jac, m->device, "jac")))
        return rc;
    if (dydt && (rc = check_device_ptr(dydt, m->device, "dydt"))) return rc;
    const pj::LaunchCfg &c = m->jac_cfg;
    if (c.groups < 1)
        return fail(PJ_EUNSUPPORTED, "one state's working set does not fit in shared memory for this model");
    pj::KParams p{};
    p.m = m->dev;
    p.sc = pj::make_scratch(m->dev, true, c.wps);
    p.n = n;
    p.T = T;
    p.P = P;
    p.Y = nmol;
    p.ldy = ldn;
    p.V = V;
    p.jac = jac;
    p.ldj = ldj;
    p.dydt = dydt;
    p.ldd = ldd;
    p.groups = c.groups;
    p.shared_const = pj::shared_const_doubles(m->N);
    DeviceProps dp = device_props(m->device);
    long long need = (n + c.groups - 1) / c.groups;
    int blocks = int(std::min<long long>(need, (long long)dp.sms * c.ctas_per_sm));
    const size_t smem = smem_bytes(m, true, c);
    cudaError_t e;
    if (const void *sk = pj::spec_conc_kernel(m, c)) {       // the model's specialised kernel
        e = cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        void *args[] = {&p};
        if (e == cudaSuccess)
            e = cudaLaunchKernel(sk, dim3(blocks), dim3(c.wps * 32 * c.groups), args, smem,
                                 static_cast<cudaStream_t>(stream));
    } else {
        e = pj::launch_conc(p, c.wps, blocks, smem, static_cast<cudaStream_t>(stream));
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return PJ_OK;
}

int pj_set_launch(pj_mech *m, int which, const pj_launch *cfg) {
    if (!m || !cfg || (which != 0 && which != 1)) return fail(PJ_EINVAL, "pj_set_launch: bad argument");
    pj::LaunchCfg c;
    c.wps = cfg->warps_per_state;
    c.groups = cfg->states_per_cta;
    c.ctas_per_sm = cfg->ctas_per_sm;
    if (!valid_shape(c)) return fail(PJ_EINVAL, "pj_set_launch: launch shape outside the supported limits");
    if (smem_bytes(m, which == 0, c) > size_t(device_props(m->device).smem_optin))
        return fail(PJ_EINVAL, "pj_set_launch: shape needs more shared memory than one CTA can have");
    (which == 0 ? m->jac_cfg : m->dydt_cfg) = c;
    return PJ_OK;
}

int pj_mech_specialize(pj_mech *m, int enable) {
    if (!m) return fail(PJ_EINVAL, "pj_mech_specialize: null model");
    if (!enable) {
        pj::spec_release(m);
        return PJ_OK;
    }
    int rc = check_model_device(m);
    if (rc) return rc;
    std::string err;
    rc = pj::specialize(m, &err);
    return rc ? fail(rc, "pj_mech_specialize: " + err) : PJ_OK;
}

int pj_mech_spec_info(const pj_mech *m, int *active_jacobian, int *active_dydt, double *compile_seconds,
                      size_t *cubin_bytes) {
    if (!m) return fail(PJ_EINVAL, "pj_mech_spec_info: null model");
    if (active_jacobian) *active_jacobian = pj::spec_kernel(m, true, false, m->jac_cfg) != nullptr;
    if (active_dydt) *active_dydt = pj::spec_kernel(m, false, false, m->dydt_cfg) != nullptr;
    if (compile_seconds) *compile_seconds = m->spec ? m->spec->compile_seconds : 0.0;
    if (cubin_bytes) *cubin_bytes = m->spec ? m->spec->cubin_bytes : 0;
    return PJ_OK;
}

int pj_get_launch(const pj_mech *m, int which, pj_launch *cfg) {
    if (!m || !cfg || (which != 0 && which != 1)) return fail(PJ_EINVAL, "pj_get_launch: bad argument");
    const pj::LaunchCfg &c = which == 0 ? m->jac_cfg : m->dydt_cfg;
    cfg->warps_per_state = c.wps;
    cfg->states_per_cta = c.groups;
    cfg->ctas_per_sm = c.ctas_per_sm;
    return PJ_OK;
}

int pj_launch_smem_bytes(const pj_mech *m, int which, const pj_launch *cfg, size_t *bytes) {
    if (!m || !cfg || !bytes || (which != 0 && which != 1)) return fail(PJ_EINVAL, "pj_launch_smem_bytes: bad argument");
    pj::LaunchCfg c;
    c.wps = cfg->warps_per_state;
    c.groups = cfg->states_per_cta;
    c.ctas_per_sm = cfg->ctas_per_sm;
    if (!valid_shape(c)) return fail(PJ_EINVAL, "pj_launch_smem_bytes: launch shape outside the supported limits");
    *bytes = smem_bytes(m, which == 0, c);
    return PJ_OK;
}

}  // extern "C"
