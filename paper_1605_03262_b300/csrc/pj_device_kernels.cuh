// sm_103a device code: batched FP64 chemical source terms and analytical Jacobian (constant
// pressure, and constant volume through the CV template flag). Included by pj_kernels.cu and by
// the runtime-compiled specialised kernels (pj_nvrtc.cu).
//
// Method (paper Sections 2-4). Per state (T, P, Y_1..Y_N) with Y_N taken as given, column j of the
// Jacobian (j = 1..N-1) is the derivative D_j = d/dY_j - d/dY_N at fixed T and P; column N is zero.
// With Delta_j = 1/W_j - 1/W_N the Section 3.1 derivatives give, for every reaction i,
//   D_j [X_l] = -[X_l] W Delta_j + (delta_lj - delta_lN) rho / W_l,
//   D_j R_i   = -W Delta_j sigma_i + rho (G_ij / W_j - G_iN / W_N),
//       sigma_i = (sum nu') R_f - (sum nu'') R_r,   G_il = k_f dPi'/d[X_l] - k_r dPi''/d[X_l],
//   D_j c_i   = psi_i D_j [M]_i,  psi_i = dc_i/d[M]_i,
//   D_j [M]_i = -W Delta_j E_i + rho (eps_ij / W_j - eps_iN / W_N),
//       eps_il = alpha_il - 1 and E_i = [M]_i - p/(RT) for the mixture (dp/dY_j = 0, Appendix B),
//       eps_il = delta_lm and E_i = [X_m] for a single third-body species m.
// Hence D_j q_i = Delta_j a_i + rho (b'_ij / W_j - b'_iN / W_N) with
//   a_i = -W (c_i sigma_i + psi_i R_i E_i),   b'_il = c_i G_il + psi_i R_i eps_il,
// and Eq. e:jac_spec becomes, for species rows k,
//   J_{k,j} = A_k Delta_j + C_k + Sparse_{k,j},
//   A_k = (W_k/rho) (sum_i nu_ki a_i + W omega_k),  Sparse_{k,j} = (W_k/W_j) sum_i nu_ki b'_ij,
//   C_k = -Sparse_{k,N}.
// The temperature column is J_{k,0} = (W_k/rho) sum_i nu_ki theta_i with
// theta_i = dq_i/dT + q_i/T (the paper's Theta_dT times rho, Eq. e:jac_temperature_update).
// The energy row (Eq. e:jac_dt) uses sum_k h_k J_{k,j} = HA Delta_j + HS_j - HS_N with
// HA = sum_k h_k A_k and HS_j = (1/W_j) sum_i dH_i b'_ij, dH_i = sum_k nu_ki H_k.
// This is the paper's Algorithm 2 reuse: every per-reaction product is formed once (reaction
// stage), scattered to species by static gather lists (gather stage), and the dense (N+1)^2
// block is written at one FMA per entry plus the reaction-local sparse terms (row stage).
//
// Parallel layout: a "group" of WPS warps evaluates one state at a time; a CTA holds several
// groups and loops persistently over rounds of states, one per group. The reaction stage of a
// round runs over the whole CTA, transposed (reaction-major, state-minor), so that small reaction
// classes still fill warps with one code path. All of a state's intermediates live in shared
// memory. Every sum has a fixed order (32-lane reductions, one lane per schedule entry), so the
// result of a state is bitwise independent of the launch shape.
#pragma once

#include "pj_device.h"

namespace pj {

constexpr double kInvLn10 = 0.43429448190325182765;
constexpr double kLn10 = 2.30258509299404568402;

__device__ __forceinline__ double warp_sum(double v) {
    // xor butterfly: a + b is commutative, so every lane ends with the same bits
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Two and four sums at once, each with exactly the addition tree of warp_sum (offsets 16, 8, 4, 2,
// 1; a + b is commutative, so each result has the same bits): in the first steps a lane keeps only
// the sums its half (quarter) of the warp finishes and trades the others with its partner, so the
// four sums cost 6 FP64 adds instead of 20. Every lane gets every sum.
__device__ __forceinline__ void warp_sum2(double &a, double &b) {
    const int lane = threadIdx.x & 31;
    const bool lo = lane < 16;
    double v = (lo ? a : b) + __shfl_xor_sync(0xffffffffu, lo ? b : a, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    a = __shfl_sync(0xffffffffu, v, 0);
    b = __shfl_sync(0xffffffffu, v, 16);
}

__device__ __forceinline__ void warp_sum4(double &a, double &b, double &c, double &d) {
    const int lane = threadIdx.x & 31;
    const bool lo = lane < 16;
    // step 16: lanes 0-15 keep (a, b), lanes 16-31 keep (c, d)
    double x = (lo ? a : c) + __shfl_xor_sync(0xffffffffu, lo ? c : a, 16);
    double y = (lo ? b : d) + __shfl_xor_sync(0xffffffffu, lo ? d : b, 16);
    // step 8: in each half, lanes with bit 3 clear keep the first, the others the second
    const bool first = (lane & 8) == 0;
    double v = (first ? x : y) + __shfl_xor_sync(0xffffffffu, first ? y : x, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    a = __shfl_sync(0xffffffffu, v, 0);
    b = __shfl_sync(0xffffffffu, v, 8);
    c = __shfl_sync(0xffffffffu, v, 16);
    d = __shfl_sync(0xffffffffu, v, 24);
}

// The threads that evaluate one state: group index in the CTA, thread index in the group, lane,
// warp in the group, warps per group (WPS template argument, or runtime when it is 0).
struct Grp {
    int grp, t, lane, wg, wps, G;
};

template <int WPS>
__device__ __forceinline__ void group_sync(const Grp &g) {
    if constexpr (WPS == 1) {
        __syncwarp();
    } else if constexpr (WPS > 1) {
        asm volatile("bar.sync %0, %1;" ::"r"(g.grp + 1), "r"(WPS * 32) : "memory");
    } else {
        if (g.wps == 1) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(g.grp + 1), "r"(g.G) : "memory");
    }
}

__device__ __forceinline__ double ipow(double x, int n) {
    double x2 = x * x;
    return n == 1 ? x : n == 2 ? x2 : n == 3 ? x2 * x : x2 * x2;
}

// n x^(n-1)
__device__ __forceinline__ double dipow(double x, int n) {
    return n == 1 ? 1.0 : n == 2 ? 2.0 * x : n == 3 ? 3.0 * x * x : 4.0 * x * x * x;
}

__device__ __forceinline__ double sel4(const double (&v)[kMaxSlots], int i) {
    return i == 0 ? v[0] : i == 1 ? v[1] : i == 2 ? v[2] : v[3];
}

// A warp's walk over chunks c0, c0 + step, ... of one schedule. Each lane takes its records of a
// chunk in order, B rows at a time, with the rows after the current batch in flight while it runs
// (with FIRST, the next chunk's first rows are requested when a chunk starts, before pre). With
// OPS the shared-memory operands of a whole batch are read (load) before any of its sums is stored
// (use), so those loads overlap instead of waiting on the stores; it costs registers, which the
// gathers (between the reaction stage and the combine) do not have to spare. pre(c) and post(c)
// run around chunk c.
template <int B, class R>
__device__ __forceinline__ void load_recs(R (&r)[B], const R *base, int x0, int len) {
#pragma unroll
    for (int u = 0; u < B; ++u) r[u] = (x0 + u < len) ? __ldg(base + 32 * (x0 + u)) : R{};
}

template <int B, bool FIRST, bool OPS, class R, class Pre, class Load, class Use, class Post>
__device__ __forceinline__ void walk(const int2 *tab, int n, int c0, int step, const R *recs, int lane, Pre &&pre,
                                     Load &&load, Use &&use, Post &&post) {
    if (c0 >= n) return;
    int2 h = __ldg(tab + c0);
    int2 hn = (c0 + step < n) ? __ldg(tab + c0 + step) : make_int2(0, 0);
    R cur[B];
    load_recs<B>(cur, recs + h.x + lane, 0, h.y);
    for (int c = c0; c < n; c += step) {
        const int2 hnn = (c + 2 * step < n) ? __ldg(tab + c + 2 * step) : make_int2(0, 0);
        R first[FIRST ? B : 1];
        if constexpr (FIRST) load_recs<B>(first, recs + hn.x + lane, 0, hn.y);
        pre(c);
        for (int x0 = 0; x0 < h.y; x0 += B) {
            R nxt[B];
            if (FIRST || x0 + B < h.y) load_recs<B>(nxt, recs + h.x + lane, x0 + B, h.y);
            else load_recs<B>(nxt, recs + hn.x + lane, 0, hn.y);      // next chunk's first rows
            if (x0 + B <= h.y) {                      // a full batch: no predicated arithmetic
                if constexpr (OPS) {
                    decltype(load(cur[0])) ops[B];
#pragma unroll
                    for (int u = 0; u < B; ++u) ops[u] = load(cur[u]);
#pragma unroll
                    for (int u = 0; u < B; ++u) use(cur[u], ops[u]);
                } else {
#pragma unroll
                    for (int u = 0; u < B; ++u) use(cur[u], load(cur[u]));
                }
            } else {
                // the chunk's last, partial batch: a loop over the remaining items (the window
                // shifts down), so that no FP64 instruction of a missing item is issued with every
                // lane predicated off; those would take FP64 pipe time like real ones
#pragma unroll 1
                for (int rem = h.y - x0; rem > 0; --rem) {
                    use(cur[0], load(cur[0]));
#pragma unroll
                    for (int u = 0; u + 1 < B; ++u) cur[u] = cur[u + 1];
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) cur[u] = nxt[u];
        }
        post(c);
        if constexpr (FIRST) {
#pragma unroll
            for (int u = 0; u < B; ++u) cur[u] = first[u];
        } else if (h.y == 0) {
            load_recs<B>(cur, recs + hn.x + lane, 0, hn.y);
        }
        h = hn;
        hn = hnn;
    }
}

__device__ __forceinline__ void no_op(int) {}

constexpr int GB = 8, HB = 4, SB = 4;           // record rows per batch: species gather, column sums and C_k, rows
constexpr unsigned kFirstItem = 0x40000000u;    // first item of a sum (coefficient records)
constexpr unsigned kPartialItem = 0x20000000u;  // a later piece of a split row entry

struct Ops4 {
    double nu, q, th, a;
};

struct StateScalars {
    double T, invT, lnT, P, lnP, W, rho, Ctot;
};

// Thermodynamics of species k (Eqs. e:cpk, e:hk; B_k and dB_k/dT of Sections 2.3.1, 3.1).
struct Thermo {
    double cpR, HR, B, dB, dcpR;
};

template <bool JAC>
__device__ __forceinline__ Thermo species_thermo(const DevModel &m, int k, double T, double invT, double lnT) {
    const double *t = m.thermo + size_t(k) * kThermoStride + (T < __ldg(m.Tmid + k) ? 0 : 18);
    const double a0 = __ldg(t + 0), a1 = __ldg(t + 1), a2 = __ldg(t + 2), a3 = __ldg(t + 3), a4 = __ldg(t + 4),
                 a5 = __ldg(t + 5);
    const double h1 = __ldg(t + 7), h2 = __ldg(t + 8), h3 = __ldg(t + 9), h4 = __ldg(t + 10);
    const double g2 = __ldg(t + 11), g3 = __ldg(t + 12), g4 = __ldg(t + 13), b0 = __ldg(t + 17);
    Thermo o;
    o.cpR = fma(T, fma(T, fma(T, fma(T, a4, a3), a2), a1), a0);
    o.HR = fma(T, fma(T, fma(T, fma(T, fma(T, h4, h3), h2), h1), a0), a5);
    o.B = fma(a0 - 1.0, lnT, b0) + T * fma(T, fma(T, fma(T, g4, g3), g2), h1) - a5 * invT;
    if constexpr (JAC) {
        const double d2 = __ldg(t + 14), d3 = __ldg(t + 15), d4 = __ldg(t + 16);
        o.dB = fma(a5, invT, a0 - 1.0) * invT + fma(T, fma(T, fma(T, h4, h3), h2), h1);
        o.dcpR = fma(T, fma(T, fma(T, d4, d3), d2), a1);
    } else {
        o.dB = 0.0;
        o.dcpR = 0.0;
    }
    return o;
}

// Third-body concentration [M]_i and E_i = [M]_i - u p/(RT) (u = 1 mixture, 0 single species).
__device__ __forceinline__ void third_body(const DevModel &m, const RxnDev &d, const double *C, double Ctot,
                                           double &M, double &E) {
    if (d.tbmode == kTbSpecies) {
        M = C[d.tbsp];
        E = M;
    } else {
        double e = 0.0;
        for (int x = 0; x < d.neff; ++x) e = fma(__ldg(m.eff_eps + d.eff_off + x), C[__ldg(m.eff_sp + d.eff_off + x)], e);
        E = e;
        M = Ctot + e;
    }
}

// One side of a reaction: the concentration product P = prod [X]^nu, its partial derivatives
// S_x = dP/d[X_x] (formed from the other factors, never by dividing by [X], Section 3.1), and the
// side's sums of nu B_k, nu dB_k/dT (equilibrium constant, Section 2.3.1) and nu H_k (energy row).
struct Side {
    double P, S[kMaxSlots], sB, sdB, sH;
};

template <int NS, bool JAC, bool UNIT>
__device__ __forceinline__ void side(const int16_t *sp, const int8_t *nu, const double *C, const double *B,
                                     const double *dB, const double *H, const double *sNu, bool kc, Side &o) {
    // UNIT: every coefficient of the side is 1 (flagged at load), so [X]^nu = [X] and its derivative
    // is 1: the products and partial derivatives below skip the factors d (multiplications by 1.0,
    // exact) and the per-species power branch
    double p[NS], d[NS];
    o.sB = 0.0;
    o.sdB = 0.0;
    o.sH = 0.0;
#pragma unroll
    for (int x = 0; x < NS; ++x) {
        const int k = sp[x];
        const double c = C[k];
        if constexpr (UNIT) {
            p[x] = c;
            d[x] = 1.0;
        } else {
            const int v = nu[x];
            if (v == 1) {
                p[x] = c;
                d[x] = 1.0;
            } else {
                const double c2 = c * c;
                if (v == 2) {
                    p[x] = c2;
                    d[x] = 2.0 * c;
                } else if (v == 3) {
                    p[x] = c2 * c;
                    d[x] = 3.0 * c2;
                } else {
                    p[x] = c2 * c2;
                    d[x] = 4.0 * c2 * c;
                }
            }
        }
        const double vd = UNIT ? 1.0 : sNu[nu[x] + kNuBias];
        if (kc) {
            o.sB = fma(vd, B[k], o.sB);
            if constexpr (JAC) o.sdB = fma(vd, dB[k], o.sdB);
        }
        if constexpr (JAC) o.sH = fma(vd, H[k], o.sH);
    }
    if constexpr (NS == 1) {
        o.P = p[0];
        o.S[0] = d[0];
    } else if constexpr (NS == 2) {
        o.P = p[0] * p[1];
        o.S[0] = UNIT ? p[1] : d[0] * p[1];
        o.S[1] = UNIT ? p[0] : d[1] * p[0];
    } else if constexpr (NS == 3) {
        const double p01 = p[0] * p[1];
        o.P = p01 * p[2];
        o.S[0] = UNIT ? p[1] * p[2] : d[0] * (p[1] * p[2]);
        o.S[1] = UNIT ? p[0] * p[2] : d[1] * (p[0] * p[2]);
        o.S[2] = UNIT ? p01 : d[2] * p01;
    } else {
        const double p01 = p[0] * p[1], p23 = p[2] * p[3];
        o.P = p01 * p23;
        o.S[0] = UNIT ? p[1] * p23 : d[0] * (p[1] * p23);
        o.S[1] = UNIT ? p[0] * p23 : d[1] * (p[0] * p23);
        o.S[2] = UNIT ? p[3] * p01 : d[2] * (p[3] * p01);
        o.S[3] = UNIT ? p[2] * p01 : d[3] * (p[2] * p01);
    }
}

template <bool JAC>
__device__ __forceinline__ void side_n(int n, bool unit, const int16_t *sp, const int8_t *nu, const double *C,
                                       const double *B, const double *dB, const double *H, const double *sNu, bool kc,
                                       Side &o) {
    if (unit) {
        switch (n) {
        case 1: side<1, JAC, true>(sp, nu, C, B, dB, H, sNu, kc, o); break;
        case 2: side<2, JAC, true>(sp, nu, C, B, dB, H, sNu, kc, o); break;
        case 3: side<3, JAC, true>(sp, nu, C, B, dB, H, sNu, kc, o); break;
        default: side<4, JAC, true>(sp, nu, C, B, dB, H, sNu, kc, o); break;
        }
        return;
    }
    switch (n) {
    case 1: side<1, JAC, false>(sp, nu, C, B, dB, H, sNu, kc, o); break;
    case 2: side<2, JAC, false>(sp, nu, C, B, dB, H, sNu, kc, o); break;
    case 3: side<3, JAC, false>(sp, nu, C, B, dB, H, sNu, kc, o); break;
    default: side<4, JAC, false>(sp, nu, C, B, dB, H, sNu, kc, o); break;
    }
}

// Reaction i: rate of progress q_i and, for the Jacobian, theta_i, a_i, dH_i and the b-slots.
// CV: the constant-volume form (Section 3.3), where rho is fixed instead of p: concentrations do
// not move with T, [M] of a mixture moves with Y through rho sum Y/W, and p = rho R T / W moves
// with T and Y (pressure-dependent rates see d ln p / dT = 1/T and d ln p / dY_j = W Delta_j).
template <bool JAC, bool CV = false>
__device__ __forceinline__ void reaction(const DevModel &m, int i, const StateScalars &s, const double *C,
                                         const double *B, const double *dB, const double *H, const double *sNu,
                                         double *sq, double *sth, double *sa, double *sdH, double *sb) {
    RxnDev d;
    {
        const int4 *src = reinterpret_cast<const int4 *>(m.rx + i);
        int4 *dst = reinterpret_cast<int4 *>(&d);
#pragma unroll
        for (int w = 0; w < 4; ++w) dst[w] = __ldg(src + w);
    }
    const MathTables *tb = m.tables;
    const double *par = m.par + d.par_off;
    const double T = s.T, invT = s.invT, lnT = s.lnT;
    double lnkf = 0.0, dlnkf = 0.0, kf = 0.0;
    double c = 1.0, dcdT = 0.0, psi = 0.0, E = 0.0;
    double pif = 0.0;                      // d ln k_f / d ln p (PLOG, Chebyshev; constant volume)
    int rev_off = 0;

    if (d.kind == kElem || d.kind == kThird) {
        const double lnA = __ldg(par + 0), beta = __ldg(par + 1), Ta = __ldg(par + 2);
        lnkf = fma(beta, lnT, lnA) - Ta * invT;
        dlnkf = fma(Ta, invT, beta) * invT;
        if (d.kform == kKfConst) {
            kf = __ldg(par + 3);
        } else if (d.kform == kKfIntPow) {
            double tp = 1.0, base = d.kpow >= 0 ? T : invT;
            for (int x = 0; x < (d.kpow >= 0 ? d.kpow : -d.kpow); ++x) tp *= base;
            kf = __ldg(par + 3) * tp;
        } else {
            kf = fast_exp(lnkf, tb);
        }
        rev_off = 4;
        if (d.kind == kThird) {
            double M;
            third_body(m, d, C, s.Ctot, M, E);
            c = M;
            dcdT = CV ? 0.0 : -M * invT;
            psi = 1.0;
        }
    } else if (d.kind == kFalloff || d.kind == kChem) {
        const double lnk0 = fma(__ldg(par + 1), lnT, __ldg(par + 0)) - __ldg(par + 2) * invT;
        const double lnki = fma(__ldg(par + 4), lnT, __ldg(par + 3)) - __ldg(par + 5) * invT;
        const double dlnk0 = fma(__ldg(par + 2), invT, __ldg(par + 1)) * invT;
        const double dlnki = fma(__ldg(par + 5), invT, __ldg(par + 4)) * invT;
        double M;
        third_body(m, d, C, s.Ctot, M, E);
        const double ratio = fast_exp(lnk0 - lnki, tb);
        const double Pr = ratio * M;
        double F = 1.0, phiF = 0.0, tauF = 0.0;   // F, dlnF/dlnPr, dlnF/dT at fixed Pr
        if (d.ftype == kTroe) {
            const double a = __ldg(par + 6), iT3 = __ldg(par + 7), iT1 = __ldg(par + 8), T2 = __ldg(par + 9);
            const double e3 = fast_exp(-T * iT3, tb), e1 = fast_exp(-T * iT1, tb);
            double Fc = fma(1.0 - a, e3, a * e1);
            double dFc = -(1.0 - a) * iT3 * e3 - a * iT1 * e1;
            if (d.flags & 1) {
                const double e2 = fast_exp(-T2 * invT, tb);
                Fc += e2;
                dFc = fma(T2 * invT * invT, e2, dFc);
            }
            const double lnFc = fast_log(Fc, tb), lFc = lnFc * kInvLn10;
            const double lPr = fast_log(fmax(Pr, 1e-300), tb) * kInvLn10;
            const double At = lPr - 0.67 * lFc - 0.4;
            const double Bt = 0.806 - 1.1762 * lFc - 0.14 * lPr;
            const double iB = 1.0 / Bt, r = At * iB;
            const double g = 1.0 / fma(r, r, 1.0);
            F = fast_exp(lnFc * g, tb);
            if constexpr (JAC) {
                const double g2r = -2.0 * g * g * r * iB;
                // below the P_r clamp F is constant, so its P_r derivative is zero there
                phiF = Pr < 1e-300 ? 0.0 : lnFc * g2r * fma(0.14, r, 1.0) * kInvLn10;
                const double dg_dlFc = g2r * fma(1.1762, r, -0.67);
                tauF = fma(lnFc * kInvLn10, dg_dlFc, g) * dFc / Fc;
            }
        } else if (d.ftype == kSri) {
            const double a = __ldg(par + 6), b = __ldg(par + 7), ic = __ldg(par + 8), lnd = __ldg(par + 9),
                         e = __ldg(par + 10);
            const double lPr = fast_log(fmax(Pr, 1e-300), tb) * kInvLn10;
            const double X = 1.0 / fma(lPr, lPr, 1.0);
            const double e1 = fast_exp(-b * invT, tb), e2 = fast_exp(-T * ic, tb);
            const double base = fma(a, e1, e2);
            const double lnb = fast_log(base, tb);
            F = fast_exp(fma(X, lnb, fma(e, lnT, lnd)), tb);
            if constexpr (JAC) {
                phiF = Pr < 1e-300 ? 0.0 : -2.0 * X * X * lPr * lnb * kInvLn10;
                tauF = fma(X * fma(a * b * invT * invT, e1, -ic * e2), 1.0 / base, e * invT);
            }
        }
        const double iPr1 = 1.0 / (1.0 + Pr);
        double phi;
        if (d.kind == kFalloff) {
            lnkf = lnki;
            dlnkf = dlnki;
            c = Pr * iPr1 * F;
            phi = iPr1 + phiF;
            psi = ratio * F * iPr1 * phi;
        } else {
            lnkf = lnk0;
            dlnkf = dlnk0;
            c = F * iPr1;
            phi = phiF - Pr * iPr1;
            const double Mg = M > 0.0 ? M : 1e-300;
            psi = F * iPr1 * (phiF / Mg - ratio * iPr1);
        }
        kf = fast_exp(lnkf, tb);
        dcdT = c * fma(phi, CV ? dlnk0 - dlnki : dlnk0 - dlnki - invT, tauF);
        rev_off = 11;
    } else if (d.kind == kPlog) {
        const int n = int(__ldg(par + 0));
        const double *t = par + 1;   // n x (p, ln p, ln A, beta, Ta)
        int lo = 0, hi = 0;
        double fr = 0.0, idl = 0.0;
        if (s.P <= __ldg(t + 0)) {
            lo = hi = 0;
        } else if (s.P >= __ldg(t + 5 * (n - 1))) {
            lo = hi = n - 1;
        } else {
            lo = 0;
            while (lo < n - 2 && !(s.P < __ldg(t + 5 * (lo + 1)))) ++lo;   // bounded even for NaN P
            hi = lo + 1;
            const double l1 = __ldg(t + 5 * lo + 1), l2 = __ldg(t + 5 * hi + 1);
            fr = (s.lnP - l1) / (l2 - l1);
            if constexpr (CV) idl = 1.0 / (l2 - l1);
        }
        const double *a = t + 5 * lo, *b = t + 5 * hi;
        const double lk1 = fma(__ldg(a + 3), lnT, __ldg(a + 2)) - __ldg(a + 4) * invT;
        const double lk2 = fma(__ldg(b + 3), lnT, __ldg(b + 2)) - __ldg(b + 4) * invT;
        const double d1 = fma(__ldg(a + 4), invT, __ldg(a + 3)) * invT;
        const double d2 = fma(__ldg(b + 4), invT, __ldg(b + 3)) * invT;
        lnkf = fma(lk2 - lk1, fr, lk1);
        dlnkf = fma(d2 - d1, fr, d1);
        if constexpr (CV) {
            pif = (lk2 - lk1) * idl;
            dlnkf = fma(pif, invT, dlnkf);
        }
        kf = fast_exp(lnkf, tb);
        rev_off = 1 + 5 * n;
    } else {   // Chebyshev, Eq. e:cheb; derivative via d T_n/dx = n U_{n-1}
        const int nt = int(__ldg(par + 0)), npc = int(__ldg(par + 1));
        const double Tt = (2.0 * invT - __ldg(par + 2)) * __ldg(par + 3);
        const double pt = (2.0 * s.lnP * kInvLn10 - __ldg(par + 4)) * __ldg(par + 5);
        const double *eta = par + 6;
        double lk = 0.0, dlk = 0.0, lkp = 0.0;
        double Tm1 = 0.0, T0 = 1.0;        // T_{t-1}, T_t at Tt
        double Um2 = 0.0, Um1 = 0.0;       // U_{t-2}, U_{t-1}
        for (int x = 0; x < nt; ++x) {
            double ct = 0.0, pm1 = 0.0, p0 = 1.0;
            double cpd = 0.0, um2 = 0.0, um1 = 0.0;   // sum_y eta y U_{y-1}(pt); U_{y-2}, U_{y-1}
            for (int y = 0; y < npc; ++y) {
                const double e = __ldg(eta + x * npc + y);
                ct = fma(e, p0, ct);
                const double pn = (y == 0) ? pt : 2.0 * pt * p0 - pm1;
                pm1 = p0;
                p0 = pn;
                if constexpr (CV) {
                    cpd = fma(e * sNu[y + kNuBias], um1, cpd);
                    const double un = (y == 0) ? 1.0 : (y == 1 ? 2.0 * pt : 2.0 * pt * um1 - um2);
                    um2 = um1;
                    um1 = un;
                }
            }
            lk = fma(ct, T0, lk);
            if constexpr (CV) lkp = fma(cpd, T0, lkp);
            dlk = fma(ct * sNu[x + kNuBias], Um1, dlk);
            const double Tn = (x == 0) ? Tt : 2.0 * Tt * T0 - Tm1;
            Tm1 = T0;
            T0 = Tn;
            const double Un = (x == 0) ? 1.0 : (x == 1 ? 2.0 * Tt : 2.0 * Tt * Um1 - Um2);
            Um2 = Um1;
            Um1 = Un;
        }
        lnkf = lk * kLn10;
        dlnkf = kLn10 * dlk * (-2.0 * invT * invT) * __ldg(par + 3);
        if constexpr (CV) {                // d pt / d ln p = 2 par5 / ln 10
            pif = 2.0 * lkp * __ldg(par + 5);
            dlnkf = fma(pif, invT, dlnkf);
        }
        kf = fast_exp(lnkf, tb);
        rev_off = 6 + nt * npc;
    }

    // concentration products, their partial derivatives, and the equilibrium-constant sums
    const bool kc = d.rev == kRevKc;
    Side sf, sr;
    side_n<JAC>(d.nr, d.flags & 2, d.rsp, d.rnu, C, B, dB, H, sNu, kc, sf);
    side_n<JAC>(d.np, d.flags & 4, d.psp, d.pnu, C, B, dB, H, sNu, kc, sr);
    int inf = 0, inb = 0;
#pragma unroll
    for (int x = 0; x < kMaxSlots; ++x) {
        inf += x < d.nr ? d.rnu[x] : 0;
        inb += x < d.np ? d.pnu[x] : 0;
    }
    const double nf = sNu[inf + kNuBias], nb = sNu[inb + kNuBias];

    // reverse rate coefficient (Section 2.3.1)
    double kr = 0.0, dlnkr = 0.0;
    if (kc) {
        const double lnKc = fma(sNu[inb - inf + kNuBias], m.lnPatmR, sr.sB - sf.sB);
        kr = fast_exp(lnkf - lnKc, tb);
        dlnkr = dlnkf - (sr.sdB - sf.sdB);
    } else if (d.rev == kRevExplicit) {
        const double *pr = par + rev_off;
        kr = fast_exp(fma(__ldg(pr + 1), lnT, __ldg(pr + 0)) - __ldg(pr + 2) * invT, tb);
        dlnkr = fma(__ldg(pr + 2), invT, __ldg(pr + 1)) * invT;
    }

    const double Rf = kf * sf.P, Rr = kr * sr.P, Rn = Rf - Rr;
    const bool elem = d.kind == kElem;   // c = 1, dc/dT = 0, psi = 0: the terms in c, psi, eps drop
    const double q = elem ? Rn : c * Rn;
    sq[i] = q;
    if constexpr (!JAC) return;

    // constant volume: [X] fixed as T moves, and no 1/rho factor moves with T or Y
    const double dRdT = CV ? fma(Rf, dlnkf, -Rr * dlnkr) : Rf * fma(-nf, invT, dlnkf) - Rr * fma(-nb, invT, dlnkr);
    const double sigma = fma(nf, Rf, -nb * Rr);
    sdH[i] = sr.sH - sf.sH;
    if (elem) {
        sth[i] = CV ? dRdT : fma(q, invT, dRdT);
        sa[i] = CV ? 0.0 : -s.W * sigma;
        // b'_il = k_f dP'/d[X_l] - k_r dP''/d[X_l]
        for (int x = 0; x < d.nslot; ++x) {
            const int info = __ldg(m.slot_info + d.slot_off + x);
            const int rs = ((info >> 16) & 0xff) - 1, ps = ((info >> 24) & 0xff) - 1;
            double G = 0.0;
            if (rs >= 0) G = kf * sel4(sf.S, rs);
            if (ps >= 0) G = fma(-kr, sel4(sr.S, ps), G);
            sb[d.slot_off + x] = G;
        }
        return;
    }
    if constexpr (CV) {
        // a_i: d[M]/dY_j = rho Delta_j (mixture) and d ln k / dY_j = pi W Delta_j (p-dependent)
        sth[i] = fma(dcdT, Rn, c * dRdT);
        const double pir = kc ? pif : 0.0;
        sa[i] = fma(psi * Rn, d.tbmode == kTbMix ? s.rho : 0.0, c * s.W * fma(Rf, pif, -Rr * pir));
    } else {
        sth[i] = fma(dcdT, Rn, fma(c, dRdT, q * invT));
        sa[i] = -s.W * fma(c, sigma, psi * Rn * E);
    }
    // b'_il = c (k_f dP'/d[X_l] - k_r dP''/d[X_l]) + psi R eps_il
    const double ckf = c * kf, ckr = c * kr, psiR = psi * Rn;
    for (int x = 0; x < d.nslot; ++x) {
        const int info = __ldg(m.slot_info + d.slot_off + x);
        const int rs = ((info >> 16) & 0xff) - 1, ps = ((info >> 24) & 0xff) - 1;
        double G = 0.0;
        if (rs >= 0) G = ckf * sel4(sf.S, rs);
        if (ps >= 0) G = fma(-ckr, sel4(sr.S, ps), G);
        sb[d.slot_off + x] = fma(psiR, __ldg(m.slot_eps + d.slot_off + x), G);
    }
}

// Streams len doubles from shared memory to global memory with 16-byte streaming stores where the
// global address allows it (head and tail peeled).
__device__ __forceinline__ void store_segment(double *g, const double *sbuf, int len, int lane) {
    const int head = (reinterpret_cast<uintptr_t>(g) & 15) ? 1 : 0;
    if (head && lane == 0 && len > 0) __stcs(g, sbuf[0]);
    const int rem = len - head;
    const int npairs = rem > 0 ? rem >> 1 : 0;
    double2 *g2 = reinterpret_cast<double2 *>(g + head);
    for (int x = lane; x < npairs; x += 32) {
        double2 v;
        v.x = sbuf[head + 2 * x];
        v.y = sbuf[head + 2 * x + 1];
        __stcs(g2 + x, v);
    }
    if (rem > 0 && (rem & 1) && lane == 0) __stcs(g + len - 1, sbuf[len - 1]);
}

using StateIO = BatchIO;

// The CTA's slice of the model image into L2 (one bulk prefetch by one thread, no completion to wait
// for): issued at kernel start, the image is L2-resident before the first stage that reads it, so
// that the first touches of its records do not each wait on DRAM. Launches of one or two rounds
// only: after an L2 flush the 13-species batch (one round) ran 41.0 instead of 38.9 us without it,
// while on many rounds the first touches are amortised and the prefetch of a large image cost the
// 360-species model 0.6 %.
__device__ __forceinline__ void prefetch_model_slice(const DevModel &m) {
    if (threadIdx.x != 0) return;
    const long long per = ((m.image_bytes + gridDim.x - 1) / gridDim.x + 15) & ~15LL;
    const long long off = per * blockIdx.x;
    if (off >= m.image_bytes) return;
    const long long len = min(per, m.image_bytes - off);
    if (len > 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(m.image + off), "r"(unsigned(len)) : "memory");
}

// Per-CTA constants of a model: Delta_j, 1/W_j and the coefficient table nu = code - kNuBias.
__device__ __forceinline__ void load_model_consts(const DevModel &m, double *smem) {
    double *sNu = smem, *sDelta = smem + 128, *sInvW = smem + 128 + m.N;
    for (int k = threadIdx.x; k < m.N; k += blockDim.x) {
        sDelta[k] = __ldg(m.Delta + k);
        sInvW[k] = __ldg(m.invW + k);
    }
    for (int c = threadIdx.x; c < 128; c += blockDim.x) sNu[c] = double(c - kNuBias);
}

// Neutral elements read by padded schedule items; written once, never overwritten by a state.
template <bool JAC>
__device__ __forceinline__ void init_neutral(const DevModel &m, const Scratch &sc, double *S, int t) {
    if (t == 0) {
        S[sc.q + m.R] = 0.0;
        if (JAC) {
            S[sc.th + m.R] = 0.0;
            S[sc.a + m.R] = 0.0;
            S[sc.dH + m.R] = 0.0;
            S[sc.b + m.nslot] = 0.0;
        }
    }
}

// Per-state scalars of a round: each is computed once per state, by thread x of the CTA for the
// round's state x, and read by the state's group from its scalar block (sc.scal). Computed in the
// group instead, every warp of the group would issue the same FP64 operations (divisions, logs)
// again: on a GPU whose FP64 pipe binds, that repetition cost about 8 % of the Jacobian's issue
// slots with two-warp groups and more with wider ones.
enum ScalarSlot : int {
    kST = 0, kSinvT, kSlnT, kSP, kSlnP, kSW, kSrho, kSCtot,   // read by the reaction stage as a block
    kSinvrho, kScp, kSdcpdT, kSinvcp, kSJ00, kSe0, kSHf, kSNumScalars
};
// Group sums the CTA-wide scalar steps read (sc.red): sum Y/W, c_p, dc_p/dT, rho (concentration
// basis), then the energy sums HA, Hf, HJ0, CF.
enum RedSlot : int { kRsYW = 0, kRcp, kRdcp, kRrho, kRHA, kRHf, kRHJ0, kRCF };

// Step 1 of a round (all threads of the CTA): T, 1/T, ln T and p (rho at constant volume) of every
// state of the round. base: the round's first state; gact: its states.
template <bool CV>
__device__ __forceinline__ void round_scalars_in(const DevModel &m, const Scratch &sc, const StateIO &io,
                                                 long long base, int gact, double *S0, int stride) {
    const int x = threadIdx.x;
    if (x < gact) {
        double *o = S0 + size_t(x) * stride + sc.scal;
        const long long st = base + x;
        const double T = __ldg(io.T + st);
        o[kST] = T;
        o[kSinvT] = 1.0 / T;
        o[kSlnT] = fast_log(T, m.tables);
        o[CV ? kSrho : kSP] = __ldg(io.P + st);
    }
    __syncthreads();
}

// Step 2 (all threads): the mixture scalars from the group sums (Section 2.1): W = 1/sum(Y/W), [M]
// (Ctot) = p/(RT) or, at constant volume, rho sum(Y/W) with p = Ctot R T, rho, ln p and 1/rho.
template <bool CV, bool CONC>
__device__ __forceinline__ void round_scalars_mix(const DevModel &m, const Scratch &sc, int gact, double *S0,
                                                  int stride) {
    __syncthreads();                                    // the groups' sums are in place
    const int x = threadIdx.x;
    if (x < gact) {
        double *o = S0 + size_t(x) * stride + sc.scal;
        const double *r = S0 + size_t(x) * stride + sc.red;
        const double sYW = r[kRsYW], T = o[kST];
        o[kSW] = 1.0 / sYW;
        o[kScp] = r[kRcp];
        o[kSdcpdT] = r[kRdcp];
        if constexpr (CV) {                                 // p = rho R T / W (Eq. e:state)
            o[kSCtot] = o[kSrho] * sYW;
            o[kSP] = o[kSCtot] * kR * T;
        } else if constexpr (CONC) {
            o[kSCtot] = o[kSP] / (kR * T);
            o[kSrho] = r[kRrho];
        } else {
            o[kSCtot] = o[kSP] / (kR * T);
            o[kSrho] = o[kSCtot] * o[kSW];
        }
        o[kSlnP] = fast_log(o[kSP], m.tables);
        o[kSinvrho] = 1.0 / o[kSrho];
        o[kSinvcp] = 1.0 / o[kScp];
    }
    __syncthreads();
}

// The scalars of one state (after step 2), as the reaction stage and the gathers use them.
__device__ __forceinline__ StateScalars load_scalars(const double *o) {
    StateScalars s;
    s.T = o[kST], s.invT = o[kSinvT], s.lnT = o[kSlnT], s.P = o[kSP], s.lnP = o[kSlnP], s.W = o[kSW];
    s.rho = o[kSrho], s.Ctot = o[kSCtot];
    return s;
}

// State prep and thermodynamics (Sections 2.1-2.2), called by every thread of the CTA (active:
// the thread's group has a state this round): Y, c_p,k, H_k, B_k (and derivatives) of every
// species, the mixture sums, the round's scalars and the concentrations. CV: the input is rho
// instead of p, and the energy arrays hold c_v,k = c_p,k - R/W_k and the molar internal energy
// U_k = H_k - R T (Section 3.3), so that the energy row below is the constant-volume one.
// CONC: the molar-concentration basis at constant pressure; the input is (T, P, V, n_1..n_{N-1}),
// [X_k] = n_k / V and [X_N] = P / (R T) - sum_{k<N} [X_k] by the ideal-gas law.
template <bool JAC, int WPS, bool CV = false, bool CONC = false>
__device__ __forceinline__ void state_prep(const DevModel &m, const Scratch &sc, double *S, const double *smem_const,
                                           const StateIO &io, long long st, const Grp &g, bool active, int gact,
                                           double *S0, int stride) {
    const int N = m.N;
    const int G = WPS ? WPS * 32 : g.G, NW = WPS ? WPS : g.wps;
    const int t = g.t, lane = g.lane, wg = g.wg;
    const double *sInvW = smem_const + 128 + N;
    double *sC = S + sc.C, *sB = S + sc.B, *sdB = S + sc.dB, *sH = S + sc.H, *scp = S + sc.cpk;
    double *sJk0 = S + sc.Jk0, *sf = S + sc.f, *sred = S + sc.red;
    const double *o = S + sc.scal;
    round_scalars_in<CV>(m, sc, io, st - g.grp, gact, S0, stride);
    double *sY = sf;   // Y parks in the f array until the concentrations exist
    if (active) {
        // ---- state prep and thermodynamics (Sections 2.1-2.2) ----
        const double T = o[kST], invT = o[kSinvT], lnT = o[kSlnT];
        const double *Ys = io.Y + st * io.ldy;
        if constexpr (CONC) {
            // every warp forms the sums in the same lane order, so all hold the same bits
            const double Ctot = o[kSP] / (kR * T);
            const double invV = 1.0 / __ldg(io.V + st);
            double sx = 0.0;
            for (int k = lane; k < N - 1; k += 32) sx += __ldg(Ys + k) * invV;
            sx = warp_sum(sx);
            for (int k = t; k < N; k += G) sC[k] = k < N - 1 ? __ldg(Ys + k) * invV : Ctot - sx;
            group_sync<WPS>(g);
            double rho_c = 0.0;
            for (int k = lane; k < N; k += 32) rho_c = fma(sC[k], __ldg(m.W + k), rho_c);
            rho_c = warp_sum(rho_c);
            if (t == 0) sred[kRrho] = rho_c;
            const double irho = 1.0 / rho_c;
            for (int k = t; k < N; k += G) sY[k] = sC[k] * __ldg(m.W + k) * irho;
        } else {
            for (int k = t; k < N; k += G) sY[k] = __ldg(Ys + k);
        }
        for (int k = t; k < N; k += G) {
            const Thermo th = species_thermo<JAC>(m, k, T, invT, lnT);
            scp[k] = kR * sInvW[k] * (CV ? th.cpR - 1.0 : th.cpR);
            sH[k] = kR * (CV ? th.HR - T : th.HR);
            sB[k] = th.B;
            if constexpr (JAC) {
                sdB[k] = th.dB;
                sJk0[k] = kR * sInvW[k] * th.dcpR;   // dcp_k/dT parks in the J_k0 array
            }
        }
        group_sync<WPS>(g);
        // species sums sum Y/W, sum Y cp_k, sum Y dcp_k/dT in a fixed 32-lane order: a one-warp group
        // computes all three; in wider groups warp w computes every NW-th sum (same order, same bits)
        if (NW == 1) {
            double r1 = 0.0, r2 = 0.0, r3 = 0.0;
            for (int k = lane; k < N; k += 32) {
                const double y = sY[k];
                r1 = fma(y, sInvW[k], r1);
                r2 = fma(y, scp[k], r2);
                if constexpr (JAC) r3 = fma(y, sJk0[k], r3);
            }
            double r4 = 0.0;
            warp_sum4(r1, r2, r3, r4);
            if (lane == 0) {
                sred[kRsYW] = r1;
                sred[kRcp] = r2;
                sred[kRdcp] = JAC ? r3 : 0.0;
            }
        } else if (JAC && NW == 2 && wg == 0) {             // warp 0: sums 0 and 2, reduced together
            double r = 0.0, u = 0.0;
            for (int k = lane; k < N; k += 32) {
                const double y = sY[k];
                r = fma(y, sInvW[k], r);
                u = fma(y, sJk0[k], u);
            }
            warp_sum2(r, u);
            if (lane == 0) {
                sred[kRsYW] = r;
                sred[kRdcp] = u;
            }
        } else {
            for (int q = wg; q < (JAC ? 3 : 2); q += NW) {
                const double *xs = q == 0 ? sInvW : q == 1 ? scp : sJk0;
                double r = 0.0;
                for (int k = lane; k < N; k += 32) r = fma(sY[k], xs[k], r);
                r = warp_sum(r);
                if (lane == 0) sred[q] = r;
            }
            if (!JAC && wg == 0 && lane == 0) sred[kRdcp] = 0.0;
        }
    }
    round_scalars_mix<CV, CONC>(m, sc, gact, S0, stride);
    if (active && !CONC) {
        const double rho = o[kSrho];
        for (int k = t; k < N; k += G) sC[k] = rho * sY[k] * sInvW[k];
    }
    // the reaction stage that follows starts with a CTA barrier
}

// Molar-concentration basis at constant pressure: state (T, V, n_1..n_{N-1}) at fixed P, with
// dT/dt (Eq. e:dTdt), dV/dt = V (dT/dt / T + (R T / P) sum_k omega_k) (the ideal-gas law at fixed
// P) and dn_k/dt = V omega_k. Its Jacobian reuses the constant-pressure reaction stage and gathers:
// with D_kl = d omega_k / d[X_l] = sum_i nu_ki b'_il at fixed T and [M] = P / (R T),
//   d(dn_k/dt)/dn_j = D_kj - D_kN,
//   d(dn_k/dt)/dV   = omega_k + G_k / W + [M] D_kN   (G_k = sum_i nu_ki a_i, a_i = -W (c sigma + psi R E)),
//   d(dn_k/dt)/dT   = V (Theta_k - (d(dn_k/dt)/dV) / T)   (Theta_k = sum_i nu_ki theta_i),
// and the T and V rows from the column sums sum_k H_k D_kj (HS_j) and sum_k D_kj (NS_j). The output
// is CSR values per state, rows in state order: the dense T and V rows, then species row k with its
// T and V entries and the columns n_j of its pattern (cc_ptr / cc_col). This function writes the T
// and V rows and the source terms, and leaves each species row's constants for the row stage in the
// gather arrays: J_k0 <- its T entry, A_k <- its V entry, C_k <- W_N C_k, so that the row stage's
// fill C_k W_N / W_j plus the sparse schedule's (W_k / W_j) nu_ki b'_ij stage (W_k / W_j) (D_kj - D_kN).
template <int WPS>
__device__ __forceinline__ void conc_tv(const DevModel &m, const Scratch &sc, double *S, const double *smem_const,
                                     const StateIO &io, long long st, const Grp &g, const StateScalars &s,
                                     double cp, double J00, double HA, double Hf) {
    const int N = m.N;
    const int G = WPS ? WPS * 32 : g.G, NW = WPS ? WPS : g.wps;
    const int t = g.t, lane = g.lane, wg = g.wg;
    const double *sInvW = smem_const + 128 + N;
    const double *scp = S + sc.cpk, *sf = S + sc.f, *sHS = S + sc.HS, *sb = S + sc.b;
    double *sJk0 = S + sc.Jk0, *sA = S + sc.A, *sCk = S + sc.Ck;
    // NS_j = sum_k D_kj = sum_i dnu_i b'_ij: the column-sum schedule of HS_j with dnu_i in place of
    // dH_i; pieces' partials where the gather partials were, then each column's pieces in order.
    // The partial and NS arrays lie in the row-staging area, free until the row stage.
    double *sNS = S + sc.part, *npart = S + sc.part + 3 * m.ngp;   // ngp >= N: no overlap
    {
        double acc = 0.0;
        walk<HB, false, false>(m.h_chunk, m.nh, wg, NW, m.h_rec, lane, no_op,
             [&](const uint4 &r) { return make_double2(__ldg(m.rx_dnu + r.z), sb[r.x & 0xffffff]); },
             [&](const uint4 &r, const double2 &o) {
                 acc = fma(o.x, o.y, acc);
                 if (r.x >> 31) {
                     npart[r.y] = acc;
                     acc = 0.0;
                 }
             },
             no_op);
    }
    group_sync<WPS>(g);
    for (int j = t; j < N; j += G) {
        double v = 0.0;
        for (int q = __ldg(m.h_pfirst + j); q < __ldg(m.h_pfirst + j + 1); ++q) v += npart[q];
        sNS[j] = v;
    }
    // SA = sum_k A_k / W_k, SF = sum_k f_k / W_k, SJ = sum_k J_k0 / W_k (every warp, same order)
    double SA = 0.0, SF = 0.0, SJ = 0.0, unused = 0.0;
    for (int k = lane; k < N; k += 32) {
        SA = fma(sA[k], sInvW[k], SA);
        SF = fma(sf[k], sInvW[k], SF);
        SJ = fma(sJk0[k], sInvW[k], SJ);
    }
    warp_sum4(SA, SF, SJ, unused);
    group_sync<WPS>(g);
    const double V = __ldg(io.V + st), invT = s.invT, M = s.Ctot, W = s.W, rho = s.rho;
    const double invcp = 1.0 / cp, WN = __ldg(m.W + N - 1);
    const double fT = -Hf * invcp;
    const double HSN = sHS[N - 1], NSN = sNS[N - 1], cpN = scp[N - 1];
    const double Z = fma(fT * WN, cpN, fma(WN, HSN, HA));
    const double iWcp = invcp / W;
    const double JTT = fma(Z * invT, iWcp, J00);
    const double invV = 1.0 / V, invM = 1.0 / M;
    const double JTV = -Z * iWcp * invV;
    const double JVV = fT * invT + V * invT * JTV + (SA + NSN);
    const double JVT = V * (JTT * invT - fT * invT * invT + W * SF * invT + W * SJ - (SA + NSN) * invT);
    const double eT = -invcp * invV / rho;
    double *out = io.jac + st * io.ldj;
    const int ld = N + 1;
    for (int x = t; x < 2 * ld; x += G) {               // T and V rows (dense)
        const int row = x >= ld, col = x - row * ld;
        double v;
        if (col < 2) {
            v = row ? (col ? JVV : JVT) : (col ? JTV : JTT);
        } else {
            const int j = col - 2;
            const double Wj = __ldg(m.W + j);
            const double jt = eT * (fma(Wj, sHS[j], -WN * HSN) + fT * (Wj * scp[j] - WN * cpN));
            v = row ? fma(V * invT, jt, (sNS[j] - NSN) * invM) : jt;
        }
        __stcs(out + x, v);
    }
    if (io.dydt) {
        double *f = io.dydt + st * io.ldd;
        for (int k = t; k <= N; k += G) {
            double v;
            if (k == 0) v = fT;
            else if (k == 1) v = V * fma(fT, invT, W * SF);
            else v = V * rho * sInvW[k - 2] * sf[k - 2];
            f[k] = v;
        }
    }
    group_sync<WPS>(g);                                 // the sums above have read A_k and J_k0
    for (int k = t; k < N; k += G) {                    // species rows' constants for the row stage
        const double iWk = sInvW[k], ck = sCk[k];
        const double DkN = -WN * iWk * ck;              // d omega_k / d[X_N]
        const double JV = M * fma(iWk, sA[k], DkN);
        sJk0[k] = V * fma(rho * iWk, sJk0[k], -JV * invT);
        sA[k] = JV;
        sCk[k] = WN * ck;
    }
    group_sync<WPS>(g);
}

// The CTA's counters: the reaction stage's next run of items, and the batched kernels' next tile.
// Declared once for the module, so that a kernel that instantiates the stages for several models
// still holds one of each in shared memory.
__shared__ int s_next_item;
__shared__ int s_slot_tile;

// One round of a CTA: each group evaluates one state (prep, gathers, rows), and the reaction stage
// of the round's states runs over the whole CTA. All threads of the CTA call this together.
// active = false: a thread without a state in this round (a group past the last state, or a
// thread outside the model's groups), which takes part in the reaction stage only. gact groups
// have states; group gg's scratch is S0 + gg * stride. CV: the constant-volume form. CONC (with
// JAC): the molar-concentration basis at constant pressure, written as sparse rows (below).
template <bool JAC, int WPS, bool CV = false, bool CONC = false>
__device__ __forceinline__ void eval_state(const DevModel &m, const Scratch &sc, double *S, const double *smem_const,
                                           const StateIO &io, long long st, const Grp &g, bool active, int gact,
                                           double *S0, int stride) {
    const int N = m.N, R = m.R;
    const int G = WPS ? WPS * 32 : g.G, NW = WPS ? WPS : g.wps;
    const int t = g.t, lane = g.lane, wg = g.wg;
    const double *sNu = smem_const, *sDelta = smem_const + 128, *sInvW = smem_const + 128 + N;
    double *sH = S + sc.H, *scp = S + sc.cpk;
    double *sJk0 = S + sc.Jk0, *sA = S + sc.A, *sCk = S + sc.Ck, *sf = S + sc.f, *sHS = S + sc.HS;
    double *sq = S + sc.q, *sth = S + sc.th, *sa = S + sc.a, *sdH = S + sc.dH, *sb = S + sc.b;
    double *spart = S + sc.part;
    (void)sHS;
    state_prep<JAC, WPS, CV, CONC>(m, sc, S, smem_const, io, st, g, active, gact, S0, stride);
    StateScalars s{};
    double cp = 0.0, dcpdT = 0.0, invrho = 0.0, invcp = 0.0;
    if (active) {                                       // (an inactive group's scratch may not exist)
        const double *o = S + sc.scal;
        s = load_scalars(o);
        cp = o[kScp], dcpdT = o[kSdcpdT], invrho = o[kSinvrho], invcp = o[kSinvcp];
    }
    double *sred = S + sc.red;
    // ---- reaction stage, all of the round's states together ----
    // Item k = (reaction i, group gg), reactions in code-path order and groups fastest: a warp's
    // lanes run a few reactions for several states, so a warp mostly takes one code path even for
    // small reaction classes. Warps take runs of 32 items from a shared counter, the costliest
    // families first, so warps that drew falloff items take fewer of the rest and the stage ends
    // balanced. The arithmetic of a reaction does not depend on who evaluates it.
    if (threadIdx.x == 0) s_next_item = blockDim.x;     // every warp's first run is its own
    __syncthreads();
    const int nitems = R * gact;
    for (int base = threadIdx.x & ~31; base < nitems;) {
        const int k = base + (threadIdx.x & 31);
        int nb = 0;
        if ((threadIdx.x & 31) == 0) nb = atomicAdd(&s_next_item, 32);
        base = __shfl_sync(0xffffffffu, nb, 0);
        if (k < nitems) {
            const int i = k / gact, gg = k - i * gact;
            double *Sg = S0 + size_t(gg) * stride;
            const StateScalars sg = load_scalars(Sg + sc.scal);
            reaction<JAC, CV>(m, i, sg, Sg + sc.C, Sg + sc.B, Sg + sc.dB, Sg + sc.H, sNu, Sg + sc.q, Sg + sc.th,
                              Sg + sc.a, Sg + sc.dH, Sg + sc.b);
        }
    }
    __syncthreads();
    if (!active) return;

    if constexpr (!JAC) {
        double w = 0.0;                                 // omega_k through the species-gather schedule
        walk<GB, false, false>(m.g_chunk, m.ng, wg, NW, m.g_rec, lane, no_op,
             [&](const uint2 &r) { return make_double2(sNu[(r.x >> 24) & 127], sq[r.x & 0xffffff]); },
             [&](const uint2 &r, const double2 &o) {
                 w = fma(o.x, o.y, w);
                 if (r.x >> 31) {
                     spart[r.y] = w;
                     w = 0.0;
                 }
             },
             no_op);
        group_sync<WPS>(g);
        for (int k = t; k < N; k += G) {                // each species: its pieces' partials, in order
            double w = 0.0;
            for (int p = __ldg(m.g_pfirst + k); p < __ldg(m.g_pfirst + k + 1); ++p) w += spart[p];
            sf[k] = __ldg(m.W + k) * invrho * w;
        }
        group_sync<WPS>(g);
        double hf = 0.0;
        for (int k = lane; k < N; k += 32) hf = fma(sH[k] * sInvW[k], sf[k], hf);
        hf = warp_sum(hf);
        double *out = io.dydt + st * io.ldd;
        for (int k = t; k <= N; k += G) out[k] = (k == 0) ? -hf * invcp : sf[k - 1];
        group_sync<WPS>(g);
        return;
    } else {
        // ---- gather stage: lane-balanced schedules (each sum is one lane's, in list order) ----
        {                                               // omega_k, J_k0, A_k
            double wq = 0.0, wt = 0.0, wa = 0.0;
            walk<GB, false, false>(m.g_chunk, m.ng, wg, NW, m.g_rec, lane, no_op,
                 [&](const uint2 &r) {
                     const int i = r.x & 0xffffff;
                     return Ops4{sNu[(r.x >> 24) & 127], sq[i], sth[i], sa[i]};
                 },
                 [&](const uint2 &r, const Ops4 &o) {
                     wq = fma(o.nu, o.q, wq);
                     wt = fma(o.nu, o.th, wt);
                     wa = fma(o.nu, o.a, wa);
                     if (r.x >> 31) {
                         double *pp = spart + 3 * r.y;   // this piece's partial slot
                         pp[0] = wq;
                         pp[1] = wt;
                         pp[2] = wa;
                         wq = wt = wa = 0.0;
                     }
                 },
                 no_op);
        }
        {                                               // HS_j = (1/W_j) sum_i dH_i b'_ij
            double acc = 0.0;
            double *hpart = spart + 3 * m.ngp;
            walk<HB, false, false>(m.h_chunk, m.nh, wg, NW, m.h_rec, lane, no_op,
                 [&](const uint4 &r) { return make_double2(sdH[r.z], sb[r.x & 0xffffff]); },
                 [&](const uint4 &r, const double2 &o) {
                     acc = fma(o.x, o.y, acc);
                     if (r.x >> 31) {
                         hpart[r.y] = acc;
                         acc = 0.0;
                     }
                 },
                 no_op);
        }
        {                                               // C_k = -(W_k/W_N) sum_i nu_ki b'_iN
            double acc = 0.0;                           // (coefficients -(W_k/W_N) nu_ki in the records)
            double *cpart = spart + 3 * m.ngp + m.nhp;
            // the last warps take the C_k chunks, which the species gather and column sums load least
            walk<HB, false, false>(m.c_chunk, m.ncc, NW - 1 - wg, NW, m.c_rec, lane, no_op,
                 [&](const uint4 &r) { return sb[r.x & 0xffffff]; },
                 [&](const uint4 &r, double b) {
                     acc = fma(__hiloint2double(int(r.w), int(r.z)), b, acc);
                     if (r.x >> 31) {
                         cpart[r.y] = acc;
                         acc = 0.0;
                     }
                 },
                 no_op);
        }
        group_sync<WPS>(g);
        // combine: each species / column sums its pieces' partials, in order
        for (int item = t; item < 3 * N; item += G) {
            if (item < N) {
                const int k = item;
                double wq = 0.0, wt = 0.0, wa = 0.0;
                for (int p = __ldg(m.g_pfirst + k); p < __ldg(m.g_pfirst + k + 1); ++p) {
                    wq += spart[3 * p];
                    wt += spart[3 * p + 1];
                    wa += spart[3 * p + 2];
                }
                const double pre = __ldg(m.W + k) * invrho;
                sf[k] = pre * wq;
                sJk0[k] = pre * wt;
                sA[k] = CV ? pre * wa : pre * fma(s.W, wq, wa);   // rho fixed: no d(1/rho)/dY term
            } else if (item < 2 * N) {
                const int j = item - N;
                double hs = 0.0;
                for (int p = __ldg(m.h_pfirst + j); p < __ldg(m.h_pfirst + j + 1); ++p) hs += spart[3 * m.ngp + p];
                sHS[j] = hs * sInvW[j];
            } else {
                const int k = item - 2 * N;
                const double *cpart = spart + 3 * m.ngp + m.nhp;
                double ck = 0.0;
                for (int p = __ldg(m.c_pfirst + k); p < __ldg(m.c_pfirst + k + 1); ++p) ck += cpart[p];
                sCk[k] = ck;
            }
        }
        group_sync<WPS>(g);
        // energy sums HA, Hf, HJ0, CF: all by a one-warp group, else every NW-th by warp w, shared
        double HA, Hf, HJ0, CF;
        if (NW == 1) {
            double x1 = 0.0, x2 = 0.0, x3 = 0.0, x4 = 0.0;
            for (int k = lane; k < N; k += 32) {
                const double hk = sH[k] * sInvW[k];
                x1 = fma(hk, sA[k], x1);
                x2 = fma(hk, sf[k], x2);
                x3 = fma(hk, sJk0[k], x3);
                x4 = fma(scp[k], sf[k], x4);
            }
            warp_sum4(x1, x2, x3, x4);
            HA = x1;
            Hf = x2;
            HJ0 = x3;
            CF = x4;
        } else {
            if (NW == 2) {                              // warp w: sums w and w + 2, reduced together
                const double *v0 = wg == 0 ? sA : sf, *v1 = wg == 0 ? sJk0 : sf;
                double x = 0.0, y = 0.0;
                for (int k = lane; k < N; k += 32) {
                    const double hk = sH[k] * sInvW[k];
                    x = fma(hk, v0[k], x);
                    y = fma(wg == 0 ? hk : scp[k], v1[k], y);
                }
                warp_sum2(x, y);
                if (lane == 0) {
                    sred[4 + wg] = x;
                    sred[6 + wg] = y;
                }
            } else {
                for (int q = wg; q < 4; q += NW) {
                    const double *v = q == 0 ? sA : q == 2 ? sJk0 : sf;
                    double x = 0.0;
                    for (int k = lane; k < N; k += 32) {
                        const double uk = q == 3 ? scp[k] : sH[k] * sInvW[k];
                        x = fma(uk, v[k], x);
                    }
                    x = warp_sum(x);
                    if (lane == 0) sred[4 + q] = x;
                }
            }
            group_sync<WPS>(g);
            HA = sred[4];
            Hf = sred[5];
            HJ0 = sred[6];
            CF = sred[7];
        }
        const double J00 = -invcp * (fma(-dcpdT * invcp, Hf, CF) + HJ0);
        const double HSN = sHS[N - 1], cpN = scp[N - 1];
        const double e0 = Hf * invcp * invcp;

        if constexpr (CONC) conc_tv<WPS>(m, sc, S, smem_const, io, st, g, s, cp, J00, HA, Hf);
        // ---- row stage: chunks of rpc rows staged per warp; dense FMA over the flattened
        //      chunk, then the chunk's lane-balanced sparse schedule, then 16-byte stores ----
        const int ld = N + 1, RPC = m.rpc;
        // the chunk's rows sit one element in when their global start is 8 mod 16, so that the
        // bulk copy to global memory has both ends 16-byte aligned
        double *const stage0 = S + sc.rows + wg * row_stride(m);
        double *stage = stage0;
        double *pbuf = stage0 + RPC * ld + 1;     // partial sums of split entries
        double *Jout = io.jac + st * io.ldj;
        constexpr int kDense = 4;
        double acc = 0.0;
        int2 comb = make_int2(0, 0);                 // this chunk's combine passes (first, count)
        int2 crec = make_int2(0, 0);                 // this lane's record of the chunk's first pass
        walk<SB, true, true>(m.s_chunk, m.n_row_chunks, wg, NW, m.s_rec, lane,
             [&](int c) {                               // dense part of chunk c
                 const int r0 = c * RPC, nel = (min(r0 + RPC, ld) - r0) * ld;
                 if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                 __syncwarp();                          // the previous chunk's bulk copy has read the stage
                 stage = stage0 + ((!CONC && (reinterpret_cast<uintptr_t>(Jout + (long long)r0 * ld) & 15)) ? 1 : 0);
                 comb = __ldg(m.s_comb_chunk + c);     // combine passes of this chunk's split entries
                 if (RPC == 1 && r0 > 0) {              // one species row: its constants once
                     const int k = r0 - 1;
                     const double a = sA[k], ck = sCk[k], jk0 = sJk0[k];
                     auto value1 = [&](int j) {
                         if constexpr (CONC) {        // T and V entries; C_k W_N / W_j elsewhere
                             const double w = (j == 0 || j == N) ? 0.0 : sInvW[j - 1];
                             return (j == 0) ? jk0 : (j == N) ? a : ck * w;
                         }
                         const double d = (j == 0 || j == N) ? 0.0 : sDelta[j - 1];
                         return (j == 0) ? jk0 : (j == N) ? 0.0 : fma(a, d, ck);
                     };
                     int x = lane;
                     for (; x - lane + 32 * kDense <= ld; x += 32 * kDense) {
                         double v[kDense];
#pragma unroll
                         for (int u = 0; u < kDense; ++u) v[u] = value1(x + 32 * u);
#pragma unroll
                         for (int u = 0; u < kDense; ++u) stage[x + 32 * u] = v[u];
                     }
                     for (; x < ld; x += 32) stage[x] = value1(x);
                     crec = comb.y > 0 ? __ldg(m.s_comb + 32 * comb.x + lane) : make_int2(0, 0);
                     __syncwarp();
                     return;
                 }
                 int x0 = lane;
                 if (r0 == 0) {                         // energy row: its own loop, so that the
                     for (int j = lane; j < ld; j += 32) {   // species rows carry no FP64 work of it
                         double v;
                         if (CONC || j == N) v = 0.0;  // (the concentration basis writes its T row itself)
                         else if (j == 0) v = J00;
                         else v = fma(-invcp, fma(HA, sDelta[j - 1], sHS[j - 1] - HSN), (scp[j - 1] - cpN) * e0);
                         stage[j] = v;
                     }
                     x0 += ld;
                 }
                 int rr = 0, j = x0;                    // (row in chunk, column) of element x
                 while (j >= ld) {
                     j -= ld;
                     ++rr;
                 }
                 auto value = [&](int rr_, int j_) {    // species row r0 + rr_ >= 1
                     const int k = r0 + rr_ - 1;
                     if constexpr (CONC) {
                         const double w = (j_ == 0 || j_ == N) ? 0.0 : sInvW[j_ - 1];
                         return (j_ == 0) ? sJk0[k] : (j_ == N) ? sA[k] : sCk[k] * w;
                     }
                     const double d = (j_ == 0 || j_ == N) ? 0.0 : sDelta[j_ - 1];
                     return (j_ == 0) ? sJk0[k] : (j_ == N) ? 0.0 : fma(sA[k], d, sCk[k]);
                 };
                 auto step = [&]() {
                     j += 32;
                     while (j >= ld) {
                         j -= ld;
                         ++rr;
                     }
                 };
                 // full batches of kDense elements per lane (loads first, then stores), then the
                 // tail one element at a time: no position is issued with every lane predicated off
                 for (; x0 - lane + 32 * kDense <= nel; x0 += 32 * kDense) {
                     double v[kDense];
#pragma unroll
                     for (int u = 0; u < kDense; ++u) {
                         v[u] = value(rr, j);
                         step();
                     }
#pragma unroll
                     for (int u = 0; u < kDense; ++u) stage[x0 + 32 * u] = v[u];
                 }
                 for (; x0 < nel; x0 += 32) {
                     stage[x0] = value(rr, j);
                     step();
                 }
                 crec = comb.y > 0 ? __ldg(m.s_comb + 32 * comb.x + lane) : make_int2(0, 0);
                 __syncwarp();
             },
             // sparse part: the chunk's lane-balanced schedule. An entry's sum starts from its dense
             // value (read at the entry's first item) and adds (W_k/W_j) nu_ki b'_ij item by item
             // (coefficients in the records), so finishing an entry is a plain store. Later pieces
             // of a split entry sum from zero into partial slots.
             [&](const uint4 &r) {
                 const bool from_dense = (r.x & (kFirstItem | kPartialItem)) == kFirstItem;
                 return make_double2(sb[r.x & 0xffffff], from_dense ? stage[r.y] : 0.0);
             },
             [&](const uint4 &r, const double2 &o) {
                 acc = (r.x & kFirstItem) ? o.y : acc;
                 acc = fma(__hiloint2double(int(r.w), int(r.z)), o.x, acc);
                 if (r.x >> 31) ((r.x & kPartialItem) ? pbuf : stage)[r.y] = acc;
             },
             [&](int c) {                               // 16-byte streaming stores of the finished rows
                 const int r0 = c * RPC, nel = (min(r0 + RPC, ld) - r0) * ld;
                 __syncwarp();
                 // split entries: each entry's segment [staged value, partial sums of its later
                 // pieces] lies on consecutive lanes of a pass and is summed by a fixed pairwise tree
                 // (lane pos adds lane pos + d when pos is a multiple of 2d), so that all lanes of the
                 // pass add at once instead of one lane per entry adding its partials in a row
                 for (int q = 0; q < comb.y; ++q) {
                     const int2 cr = q == 0 ? crec : __ldg(m.s_comb + 32 * (comb.x + q) + lane);
                     const int pos = cr.y & 255, len = (cr.y >> 8) & 255, levels = cr.y >> 16;
                     double v = 0.0;
                     if (len) v = cr.x >= 0 ? stage[cr.x] : pbuf[-1 - cr.x];
                     for (int l = 0; l < levels; ++l) {
                         const int d = 1 << l;
                         const double o = __shfl_down_sync(0xffffffffu, v, d);
                         if ((pos & (2 * d - 1)) == 0 && pos + d < len) v += o;
                     }
                     if (len && pos == 0) stage[cr.x] = v;
                 }
                 // the finished rows go out as one bulk copy (TMA engine) of their 16-byte aligned
                 // middle, issued by lane 0 after the warp's shared-memory writes are fenced for the
                 // async proxy; the odd first and last elements are plain stores
                 // (one-row chunks keep the warp's own 16-byte stores: their copy would have to be read
                 // before the next row's dense fill, measured slower)
                 if constexpr (CONC) {                  // compact the staged rows into CSR rows
                     __syncwarp();
                     for (int rr = 0; rr < RPC && r0 + rr <= N; ++rr) {
                         const int r = r0 + rr;
                         if (r == 0 || r == N) continue;
                         const int k = r - 1, e0 = __ldg(m.cc_ptr + k), len = __ldg(m.cc_ptr + k + 1) - e0;
                         const double *srow = stage + rr * ld;
                         double *o = Jout + 2 * ld + 2 * k + e0;
                         if (lane < 2) __stcs(o + lane, srow[lane ? N : 0]);
                         for (int e = lane; e < len; e += 32 * kDense) {   // loads first, then stores
                             int col[kDense];
                             double w[kDense], v[kDense];
#pragma unroll
                             for (int u = 0; u < kDense; ++u) {
                                 const bool in = e + 32 * u < len;   // a full row: column = position
                                 col[u] = !in ? 0 : len == N - 1 ? e + 32 * u : __ldg(m.cc_col + e0 + e + 32 * u);
                                 w[u] = in ? __ldg(m.cc_wr + e0 + e + 32 * u) : 0.0;
                             }
#pragma unroll
                             for (int u = 0; u < kDense; ++u) v[u] = srow[1 + col[u]];
#pragma unroll
                             for (int u = 0; u < kDense; ++u)
                                 if (e + 32 * u < len) __stcs(o + 2 + e + 32 * u, v[u] * w[u]);
                         }
                     }
                     __syncwarp();
                     return;
                 }
                 if (RPC == 1) {
                     __syncwarp();
                     store_segment(Jout + (long long)r0 * ld, stage, nel, lane);
                     __syncwarp();
                     return;
                 }
                 asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                 __syncwarp();
                 if (lane == 0) {
                     double *gdst = Jout + (long long)r0 * ld;
                     const int head = int(stage - stage0), body = (nel - head) & ~1;
                     if (head) __stcs(gdst, stage[0]);
                     if (body > 0) {
                         const unsigned saddr = unsigned(__cvta_generic_to_shared(stage + head));
                         asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                                      :: "l"(gdst + head), "r"(saddr), "r"(body * 8) : "memory");
                         asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                     }
                     if (head + body < nel) __stcs(gdst + nel - 1, stage[nel - 1]);
                 }
             });
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncwarp();                                   // the stage may be reused (gather partials)
        if (!CONC && io.dydt) {
            double *out = io.dydt + st * io.ldd;
            for (int k = t; k <= N; k += G) out[k] = (k == 0) ? -Hf * invcp : sf[k - 1];
        }
        group_sync<WPS>(g);
    }
}

// Body of the evaluation kernel: the CTA's groups loop over rounds of p.groups states. The
// runtime-specialised kernels call it with the model's sizes and offsets as constants.
template <bool JAC, int WPS, bool CV, bool CONC = false>
__device__ __forceinline__ void eval_kernel_body(const KParams &p) {
    extern __shared__ __align__(16) double smem[];
    const DevModel &m = p.m;
    Grp g;
    g.wps = WPS;
    g.G = WPS * 32;
    g.grp = threadIdx.x / g.G;
    g.t = threadIdx.x - g.grp * g.G;
    g.lane = threadIdx.x & 31;
    g.wg = g.t >> 5;
    if (p.n <= 2LL * gridDim.x * p.groups) prefetch_model_slice(m);
    load_model_consts(m, smem);
    double *S = smem + p.shared_const + size_t(g.grp) * p.sc.total;
    init_neutral<JAC>(m, p.sc, S, g.t);
    __syncthreads();
    const StateIO io{p.T, p.P, p.Y, p.ldy, p.jac, p.ldj, p.dydt, p.ldd, p.V};
    double *S0 = smem + p.shared_const;
    for (long long base = (long long)blockIdx.x * p.groups; base < p.n; base += (long long)gridDim.x * p.groups) {
        const long long st = base + g.grp;
        const int gact = int(min((long long)p.groups, p.n - base));
        eval_state<JAC, WPS, CV, CONC>(m, p.sc, S, smem, io, st, g, st < p.n, gact, S0, p.sc.total);
    }
}

template <bool JAC, int WPS, bool CV, bool CONC = false>
__global__ void __launch_bounds__(512, 1) pj_eval_kernel(const __grid_constant__ KParams p) {
    eval_kernel_body<JAC, WPS, CV, CONC>(p);
}

// States [begin, end) of one tile of the batched form, in CTA rounds of it.groups states.
template <bool JAC>
__device__ __forceinline__ void run_tile(const DevModel &m, const BatchItem &it, double *smem, long long begin,
                                         long long end, const Grp &g) {
    double *S0 = smem + it.shared_const;
    double *S = S0 + size_t(g.grp) * it.sc.total;   // used only by the model's groups
    const bool member = g.grp < it.groups;
    for (long long base = begin; base < end; base += it.groups) {
        const int gact = int(min((long long)it.groups, end - base));
        eval_state<JAC, 0>(m, it.sc, S, smem, it.io, base + g.grp, g, member && g.grp < gact, gact, S0, it.sc.total);
    }
}

// Persistent kernel over tiles of states from several models (the batched form): each CTA takes
// the next tile from an atomic counter, loads the tile's model constants when the model changes,
// and its groups evaluate the tile's states with the model's group width. The model's DevModel is
// read in place from its image (a read-only pointer), not copied into static shared memory: the
// 432-byte copy left the 360-species model's 16-warp working set no room, so plans ran that model
// at 8 warps per state (one-item plan 3.38 ms, now 2.69 ms; the other models within 0.5 %).
template <bool JAC>
__global__ void __launch_bounds__(512, 1) pj_batch_kernel(const __grid_constant__ BatchParams p) {
    extern __shared__ __align__(16) double smem[];
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) s_slot_tile = atomicAdd(p.counter, 1);
        __syncthreads();
        const int tile = s_slot_tile;
        if (tile >= p.ntiles) break;
        const BatchTile tl = p.tiles[tile];
        const BatchItem &it = p.items[tl.item];
        const DevModel *__restrict__ mp = it.m;
        Grp g;
        g.wps = it.wps;
        g.G = it.wps * 32;
        g.grp = threadIdx.x / g.G;
        g.t = threadIdx.x - g.grp * g.G;
        g.lane = threadIdx.x & 31;
        g.wg = g.t >> 5;
        double *S = smem + it.shared_const + size_t(g.grp) * it.sc.total;
        if (tl.item != cur) {
            load_model_consts(*mp, smem);
            if (g.grp < it.groups) init_neutral<JAC>(*mp, it.sc, S, g.t);
            cur = tl.item;
            __syncthreads();
        }
        run_tile<JAC>(*mp, it, smem, tl.begin, tl.begin + tl.count, g);
        __syncthreads();
    }
}

// Batched form, specialised for a plan's models (kernels generated by pj_nvrtc.cu): each (model,
// group width) pair of the plan is a slot whose sizes, offsets and width Spec supplies as
// compile-time constants, and whose DevModel (the model image's device pointers) Spec::dev() reads
// from the generated module's constant memory. Held there, like the plain kernel's parameters,
// the pointers are operands of the instructions that use them; copied from shared memory into a
// local DevModel they took registers of their own, and the one-model plan of the 360-species
// model ran 1.55 x the plain kernel's time.
template <bool JAC, int WPS, class Spec>
__device__ __forceinline__ void run_tile_spec(const BatchItem *itp, long long begin, long long end, bool fresh) {
    extern __shared__ __align__(16) double smem[];
    const BatchItem &it = *itp;
    DevModel m = Spec::dev();
    Spec::spec_model(m);
    Scratch sc;
    Spec::spec_scratch(sc);
    Grp g;
    g.wps = WPS;
    g.G = WPS * 32;
    g.grp = threadIdx.x / g.G;
    g.t = threadIdx.x - g.grp * g.G;
    g.lane = threadIdx.x & 31;
    g.wg = g.t >> 5;
    const int groups = Spec::kGroups;                   // the slot's states per round, as a constant
    double *S0 = smem + Spec::kSharedConst;
    double *S = S0 + size_t(g.grp) * sc.total;
    const bool member = g.grp < groups;
    if (fresh) {
        load_model_consts(m, smem);
        if (member) init_neutral<JAC>(m, sc, S, g.t);
        __syncthreads();
    }
    const StateIO &io = it.io;            // read in place (a local copy cost the mix 1.7 %)
    for (long long base = begin; base < end; base += groups) {
        const int gact = int(min((long long)groups, end - base));
        eval_state<JAC, WPS>(m, sc, S, smem, io, base + g.grp, g, member && g.grp < gact, gact, S0, sc.total);
    }
}

// One slot's part of the specialised batched kernel: CTAs take the slot's tiles, [first, end) of
// the plan's tile table, from the slot's counter, and evaluate them with the slot's constants.
// The kernel runs the slots' parts one after another (a CTA moves on when the slot's tiles are
// all taken, without waiting for other CTAs), each part inlined on its own: no switch or call
// between models inside the loop, so each part gets the registers of a single-model kernel.
template <bool JAC, int WPS, class Spec>
__device__ __forceinline__ void run_slot_seq(const BatchParams &p, int slot, int first, int end) {
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) s_slot_tile = first + atomicAdd(p.counter + slot, 1);
        __syncthreads();
        const int tile = s_slot_tile;
        if (tile >= end) break;
        const BatchTile tl = p.tiles[tile];
        const bool fresh = tl.item != cur;
        run_tile_spec<JAC, WPS, Spec>(p.items + tl.item, tl.begin, tl.begin + tl.count, fresh);
        cur = tl.item;
        __syncthreads();
    }
    __syncthreads();                                    // every thread has read s_slot_tile
}

}  // namespace pj
