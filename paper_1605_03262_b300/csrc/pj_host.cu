// pj_eval_jacobian_host: the end-to-end entry point on host buffers. Chunks of states are copied to
// device staging buffers, evaluated and copied back, alternating between two streams so that the
// copies of one chunk overlap the kernel of the next.
#include <algorithm>
#include <string>

#include "../../include/pyjac_b300.h"
#include "pj_internal.h"

struct pj_host_staging {
    int64_t chunk = 0;
    cudaStream_t st[2] = {nullptr, nullptr};
    double *T[2] = {nullptr, nullptr}, *P[2] = {nullptr, nullptr}, *Y[2] = {nullptr, nullptr};
    double *J[2] = {nullptr, nullptr}, *F[2] = {nullptr, nullptr};
};

void pj_host_staging_release(pj_mech *m) {
    pj_host_staging *s = m ? m->staging : nullptr;
    if (!s) return;
    for (int b = 0; b < 2; ++b) {
        if (s->st[b]) cudaStreamSynchronize(s->st[b]);
        cudaFree(s->T[b]);
        cudaFree(s->P[b]);
        cudaFree(s->Y[b]);
        cudaFree(s->J[b]);
        cudaFree(s->F[b]);
        if (s->st[b]) cudaStreamDestroy(s->st[b]);
    }
    delete s;
    m->staging = nullptr;
}

namespace {
int host_fail(int code, const std::string &msg) { return pj::set_error(code, msg); }

int cuda_err(cudaError_t e, const char *what) {
    return host_fail(PJ_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

int ensure_staging(pj_mech *m, int64_t chunk) {
    pj_host_staging *s = m->staging;
    if (s && s->chunk >= chunk) return PJ_OK;
    pj_host_staging_release(m);
    s = new (std::nothrow) pj_host_staging();
    if (!s) return host_fail(PJ_ENOMEM, "host allocation failed");
    m->staging = s;
    s->chunk = chunk;
    const size_t N = size_t(m->N), nn = (N + 1) * (N + 1);
    for (int b = 0; b < 2; ++b) {
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&s->st[b], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaMalloc(&s->T[b], chunk * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&s->P[b], chunk * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&s->Y[b], chunk * N * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&s->J[b], chunk * nn * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&s->F[b], chunk * (N + 1) * sizeof(double))) != cudaSuccess) {
            pj_host_staging_release(m);
            cudaGetLastError();
            return host_fail(e == cudaErrorMemoryAllocation ? PJ_ENOMEM : PJ_ECUDA,
                             std::string("device staging buffers: ") + cudaGetErrorString(e));
        }
    }
    return PJ_OK;
}
}  // namespace

extern "C" int pj_eval_jacobian_host(const pj_mech *cm, int64_t n, const double *T, const double *P, const double *Y,
                                     int64_t ldy, double *jac, int64_t ldj, double *dydt, int64_t ldd,
                                     int64_t chunk_states) {
    pj_mech *m = const_cast<pj_mech *>(cm);
    if (!m) return host_fail(PJ_EINVAL, "pj_eval_jacobian_host: null model");
    const int64_t N = m->N, nn = (N + 1) * (N + 1);
    if (n < 0) return host_fail(PJ_EINVAL, "pj_eval_jacobian_host: n < 0");
    if (ldy < N) return host_fail(PJ_EINVAL, "pj_eval_jacobian_host: ldy < number of species");
    if (ldj < nn) return host_fail(PJ_EINVAL, "pj_eval_jacobian_host: ldj < (number of species + 1)^2");
    if (dydt && ldd < N + 1) return host_fail(PJ_EINVAL, "pj_eval_jacobian_host: ldd < number of species + 1");
    if (n == 0) return PJ_OK;
    if (!T || !P || !Y || !jac) return host_fail(PJ_EINVAL, "pj_eval_jacobian_host: null pointer");
    // 64 MB of Jacobians per chunk: the copy stream waits only for the first chunk's kernel
    int64_t chunk = chunk_states > 0 ? chunk_states : std::max<int64_t>(1024, (64ll << 20) / (nn * 8));
    chunk = std::min(chunk, n);
    int rc = ensure_staging(m, chunk);
    if (rc) return rc;
    pj_host_staging *s = m->staging;
    const size_t d = sizeof(double);
    for (int64_t c0 = 0, it = 0; c0 < n; c0 += chunk, ++it) {
        const int b = int(it & 1);
        const int64_t cn = std::min(chunk, n - c0);
        cudaStream_t st = s->st[b];
        cudaError_t e;
        // strided host rows go by 2D copies, contiguous ones by plain copies
        if ((e = cudaMemcpyAsync(s->T[b], T + c0, cn * d, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(s->P[b], P + c0, cn * d, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = ldy == N ? cudaMemcpyAsync(s->Y[b], Y + c0 * ldy, cn * N * d, cudaMemcpyHostToDevice, st)
                          : cudaMemcpy2DAsync(s->Y[b], N * d, Y + c0 * ldy, ldy * d, N * d, cn,
                                              cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_err(e, "host-to-device copy");
        rc = pj_eval_jacobian(m, cn, s->T[b], s->P[b], s->Y[b], N, s->J[b], nn, dydt ? s->F[b] : nullptr, N + 1, st);
        if (rc) return rc;
        if ((e = ldj == nn ? cudaMemcpyAsync(jac + c0 * ldj, s->J[b], cn * nn * d, cudaMemcpyDeviceToHost, st)
                           : cudaMemcpy2DAsync(jac + c0 * ldj, ldj * d, s->J[b], nn * d, nn * d, cn,
                                               cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_err(e, "device-to-host copy");
        if (dydt && (e = cudaMemcpy2DAsync(dydt + c0 * ldd, ldd * d, s->F[b], (N + 1) * d, (N + 1) * d, cn,
                                           cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_err(e, "device-to-host copy");
    }
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = cudaStreamSynchronize(s->st[b]);
        if (e != cudaSuccess) return cuda_err(e, "stream synchronize");
    }
    return PJ_OK;
}
