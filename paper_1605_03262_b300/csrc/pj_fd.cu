// First-order forward-difference Jacobian on the GPU: the finite-difference comparison of the
// paper's performance analysis (Section 5.2: a first-order forward difference adapted from CVODE),
// built on the library's own source-term kernel.
//
// Column c of the Jacobian of state s is (f(y + h_c d_c) - f(y)) / h_c, where d_0 moves T, d_c
// (c = 1..N-1) moves Y_c by +h_c and Y_N by -h_c (the directions of the analytical columns, which
// differentiate along Y_c with Y_N = 1 - sum of the others), and column N is zero. The increment is
// h_c = 2^-26 max(|y_c|, a_c) with a_0 = 1 K and a_c = 1e-10 for mass fractions: CVODE's relative
// increment sqrt(unit roundoff) |y_c| (2^-26 is exactly the square root of the double epsilon),
// with a fixed floor in place of its error-weight term, which needs an integrator's tolerances and
// step size. The increments are exact functions of the inputs.
//
// A pass over a chunk of states: source terms at the states, a kernel that writes the N perturbed
// copies of every state, one source-term launch over all of them, and a kernel that forms the
// columns. The perturbed states and their source terms live in the caller's workspace.
#include <algorithm>

#include "pj_internal.h"

namespace pj {

__device__ __forceinline__ double fd_increment(int c, double T, const double *Y) {
    const double y = c == 0 ? T : Y[c - 1], a = c == 0 ? 1.0 : 1e-10;
    return 0x1p-26 * fmax(fabs(y), a);
}

// Perturbed copies: state s, column c < N -> row s * N + c of (Tp, Pp, Yp[N]).
__global__ void fd_perturb_kernel(int N, long long ns, const double *T, const double *P, const double *Y,
                                  long long ldy, double *Tp, double *Pp, double *Yp) {
    for (long long s = blockIdx.x; s < ns; s += gridDim.x) {
        const double *Ys = Y + s * ldy;
        const double Ts = T[s];
        for (int x = threadIdx.x; x < N * N; x += blockDim.x) {
            const int c = x / N, k = x - c * N;
            double v = Ys[k];
            if (c > 0) {
                const double h = fd_increment(c, Ts, Ys);
                if (k == c - 1) v = Ys[k] + h;
                else if (k == N - 1) v = Ys[k] - h;
            }
            Yp[(s * N + c) * N + k] = v;
        }
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            Tp[s * N + c] = c == 0 ? Ts + fd_increment(0, Ts, Ys) : Ts;
            Pp[s * N + c] = P[s];
        }
    }
}

// Columns: J[s][k][c] = (Fp[s * N + c][k] - F0[s][k]) / h_c for c < N, 0 for c = N.
__global__ void fd_difference_kernel(int N, long long ns, const double *T, const double *Y, long long ldy,
                                     const double *F0, const double *Fp, double *jac, long long ldj) {
    const int ld = N + 1;
    for (long long s = blockIdx.x; s < ns; s += gridDim.x) {
        const double *Ys = Y + s * ldy;
        const double Ts = T[s];
        for (int x = threadIdx.x; x < ld * ld; x += blockDim.x) {
            const int k = x / ld, c = x - k * ld;
            double v = 0.0;
            if (c < N) v = (Fp[(s * N + c) * ld + k] - F0[s * ld + k]) / fd_increment(c, Ts, Ys);
            jac[s * ldj + x] = v;
        }
    }
}

static int fd_blocks(long long ns) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return int(std::min<long long>(ns, (long long)sms * 8));
}

cudaError_t launch_fd_perturb(int N, long long ns, const double *T, const double *P, const double *Y, long long ldy,
                              double *Tp, double *Pp, double *Yp, cudaStream_t st) {
    if (ns <= 0) return cudaSuccess;
    fd_perturb_kernel<<<fd_blocks(ns), 256, 0, st>>>(N, ns, T, P, Y, ldy, Tp, Pp, Yp);
    return cudaGetLastError();
}

cudaError_t launch_fd_difference(int N, long long ns, const double *T, const double *Y, long long ldy,
                                 const double *F0, const double *Fp, double *jac, long long ldj, cudaStream_t st) {
    if (ns <= 0) return cudaSuccess;
    fd_difference_kernel<<<fd_blocks(ns), 256, 0, st>>>(N, ns, T, Y, ldy, F0, Fp, jac, ldj);
    return cudaGetLastError();
}

}  // namespace pj
