/*
 * Oracle: plain, slow FP64 CPU evaluation of the constant-pressure chemical source terms and their
 * analytical Jacobian, written from the paper (Niemeyer, Curtis & Sung, "pyJac", Sections 2-3).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, the smoke check and the benchmark's CPU-baseline leg may
 * load this library. It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes, per state (T, P, Y_1..Y_N), with Y_N taken as given:
 *   f  = {dT/dt, dY_1/dt, ..., dY_N/dt}                       (Eqs. e:ode, e:dTdt; N+1 entries)
 *   J  = (N+1) x (N+1), row-major, row/column 0 = temperature, rows/columns 1..N = species 1..N.
 *        Column j (1..N-1) is the derivative along Y_j with Y_N = 1 - sum_{k<N} Y_k (Eq. e:y_nsp),
 *        i.e. d/dY_j - d/dY_N; column N is identically zero (Y_N is not a state variable); row N is
 *        the paper's placeholder row for the last species (Section 3.2).
 * The Jacobian follows the chain-rule definitions of Section 3.1 term by term: per reaction the
 * derivatives dq_i/dT (via dc_i/dT, dR_i/dT) and dq_i/dY_j (via dc_i/dY_j and the concentration
 * product derivatives), then the species rows by Eq. e:jac_spec and the energy row by Eq. e:jac_dt.
 * It does not use the Section 4 reuse transformations. Sums over reactions and species use
 * Neumaier compensation. Optionally every output entry also gets a "scale" = the sum of the
 * absolute values of the terms it is made of, so that tests can tell a cancelled entry from a
 * well-conditioned one.
 *
 * Readings where the paper is silent (all shared with the CUDA path by specification, not code):
 *   - NASA7 uses the low-temperature set iff T < T_mid.
 *   - Falloff: k_f = k_inf; chemically activated: k_f = k_0; their Arrhenius parameters enter dk_f/dT.
 *   - log10 P_r is taken of max(P_r, 1e-300).
 *   - PLOG: bracket p_i <= P < p_{i+1}; outside [p_1, p_n] the end rate is used.
 *   - Species-m third-body reactions: c_i = [X_m], differentiated like a concentration.
 */
#include <complex.h>
#include <errno.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle_model.h"

/* ---------------------------------------------------------------------------------------------
 * Template instantiations of the source terms: double (compensated sums) and double complex.
 * <tgmath.h> dispatches exp/log/pow on the argument type. */
#include <tgmath.h>

#define SCALAR double
#define FN(x) x##_d
#define RE(x) (x)
#define PJO_COMPENSATED 1
#include "source_terms.inc"
#undef SCALAR
#undef FN
#undef RE
#undef PJO_COMPENSATED

#define SCALAR double complex
#define FN(x) x##_z
#define RE(x) creal(x)
#define PJO_COMPENSATED 0
#include "source_terms.inc"
#undef SCALAR
#undef FN
#undef RE
#undef PJO_COMPENSATED

#define PJO_OK 0
#define PJO_EINVAL (-1)
#define PJO_EFORMAT (-2)
#define PJO_ENOMEM (-4)

/* ---------------------------------------------------------------------------------------------
 * Reader of the binary model format. */

typedef struct { const unsigned char *p, *end; int bad; } rdr;

static void rd(rdr *r, void *dst, size_t n)
{
    if (r->bad || (size_t)(r->end - r->p) < n) { r->bad = 1; memset(dst, 0, n); return; }
    memcpy(dst, r->p, n);
    r->p += n;
}
static int rdi(rdr *r) { int v; rd(r, &v, 4); return v; }
static double rdd(rdr *r) { double v; rd(r, &v, 8); return v; }

void pjo_mech_free(pjo_mech *m)
{
    if (!m) return;
    if (m->rx) {
        for (int i = 0; i < m->nr; ++i) {
            free(m->rx[i].alpha);
            free(m->rx[i].plog);
            free(m->rx[i].eta);
        }
    }
    free(m->rx);
    free(m->W);
    free(m->Tmid);
    free(m->alo);
    free(m->ahi);
    free(m->elem);
    free(m);
}

static int add_slots(rdr *r, int n, int *sp, int *nu, int ns)
{
    if (n < 0 || n > PJO_MAXSLOT) return 0;
    for (int s = 0; s < n; ++s) {
        sp[s] = rdi(r);
        nu[s] = rdi(r);
        if (sp[s] < 0 || sp[s] >= ns || nu[s] < 1 || nu[s] > 8) return 0;
    }
    return 1;
}

int pjo_mech_load(const void *buf, size_t len, pjo_mech **out)
{
    if (!buf || !out) return PJO_EINVAL;
    *out = NULL;
    rdr r = {(const unsigned char *)buf, (const unsigned char *)buf + len, 0};
    char magic[8];
    rd(&r, magic, 8);
    if (r.bad || memcmp(magic, "PYJACMEC", 8) != 0) return PJO_EFORMAT;
    unsigned ver, ne, ns, nr;
    rd(&r, &ver, 4); rd(&r, &ne, 4); rd(&r, &ns, 4); rd(&r, &nr, 4);
    if (r.bad || ver != 1 || ns < 2 || ns > 100000 || nr > 1000000 || ne > 64) return PJO_EFORMAT;
    pjo_mech *m = calloc(1, sizeof(*m));
    if (!m) return PJO_ENOMEM;
    m->ne = (int)ne; m->ns = (int)ns; m->nr = (int)nr;
    m->W = calloc(ns, sizeof(double));
    m->Tmid = calloc(ns, sizeof(double));
    m->alo = calloc(7 * ns, sizeof(double));
    m->ahi = calloc(7 * ns, sizeof(double));
    m->elem = calloc((size_t)ns * (ne ? ne : 1), sizeof(int));
    m->rx = calloc(nr ? nr : 1, sizeof(pjo_rxn));
    if (!m->W || !m->Tmid || !m->alo || !m->ahi || !m->elem || !m->rx) { pjo_mech_free(m); return PJO_ENOMEM; }
    for (unsigned k = 0; k < ns; ++k) {
        m->W[k] = rdd(&r);
        (void)rdd(&r);
        m->Tmid[k] = rdd(&r);
        (void)rdd(&r);
        for (int c = 0; c < 7; ++c) m->alo[7 * k + c] = rdd(&r);
        for (int c = 0; c < 7; ++c) m->ahi[7 * k + c] = rdd(&r);
        for (unsigned e = 0; e < ne; ++e) m->elem[k * ne + e] = rdi(&r);
        if (r.bad || !(m->W[k] > 0.0)) { pjo_mech_free(m); return PJO_EFORMAT; }
    }
    for (unsigned i = 0; i < nr; ++i) {
        pjo_rxn *x = &m->rx[i];
        x->kind = rdi(&r);
        x->rev = rdi(&r);
        if (x->kind < 0 || x->kind > 5 || x->rev < 0 || x->rev > 2) { pjo_mech_free(m); return PJO_EFORMAT; }
        x->nr = rdi(&r);
        if (r.bad || !add_slots(&r, x->nr, x->rsp, x->rnu, (int)ns)) { pjo_mech_free(m); return PJO_EFORMAT; }
        x->np = rdi(&r);
        if (r.bad || !add_slots(&r, x->np, x->psp, x->pnu, (int)ns)) { pjo_mech_free(m); return PJO_EFORMAT; }
        x->A = rdd(&r); x->beta = rdd(&r); x->Ta = rdd(&r);
        if (x->rev == PJO_REV_EXPLICIT) { x->Ar = rdd(&r); x->betar = rdd(&r); x->Tar = rdd(&r); }
        if (x->kind == PJO_THIRD || x->kind == PJO_FALLOFF || x->kind == PJO_CHEM) {
            x->tb_mode = rdi(&r);
            x->tb_sp = rdi(&r);
            int neff = rdi(&r);
            if (r.bad || neff < 0 || neff > (int)ns || (x->tb_mode != PJO_TB_MIX && x->tb_mode != PJO_TB_SPECIES) ||
                (x->tb_mode == PJO_TB_SPECIES && (x->tb_sp < 0 || x->tb_sp >= (int)ns))) {
                pjo_mech_free(m); return PJO_EFORMAT;
            }
            if (x->tb_mode == PJO_TB_MIX) {
                x->alpha = malloc(ns * sizeof(double));
                if (!x->alpha) { pjo_mech_free(m); return PJO_ENOMEM; }
                for (unsigned k = 0; k < ns; ++k) x->alpha[k] = 1.0;
            }
            for (int e = 0; e < neff; ++e) {
                int s = rdi(&r);
                double a = rdd(&r);
                if (r.bad || s < 0 || s >= (int)ns || x->tb_mode != PJO_TB_MIX) { pjo_mech_free(m); return PJO_EFORMAT; }
                x->alpha[s] = a;
            }
        }
        if (x->kind == PJO_FALLOFF || x->kind == PJO_CHEM) {
            for (int c = 0; c < 3; ++c) x->k0[c] = rdd(&r);
            for (int c = 0; c < 3; ++c) x->kinf[c] = rdd(&r);
            x->ftype = rdi(&r);
            for (int c = 0; c < 5; ++c) x->fp[c] = rdd(&r);
            x->has_T2 = rdi(&r);
            if (r.bad || x->ftype < 0 || x->ftype > 2) { pjo_mech_free(m); return PJO_EFORMAT; }
        }
        if (x->kind == PJO_PLOG) {
            x->nplog = rdi(&r);
            if (r.bad || x->nplog < 1 || x->nplog > 64) { pjo_mech_free(m); return PJO_EFORMAT; }
            x->plog = malloc(4 * x->nplog * sizeof(double));
            if (!x->plog) { pjo_mech_free(m); return PJO_ENOMEM; }
            for (int c = 0; c < 4 * x->nplog; ++c) x->plog[c] = rdd(&r);
            for (int c = 1; c < x->nplog; ++c)
                if (!(x->plog[4 * c] > x->plog[4 * (c - 1)])) { pjo_mech_free(m); return PJO_EFORMAT; }
        }
        if (x->kind == PJO_CHEB) {
            x->nt = rdi(&r);
            x->npc = rdi(&r);
            if (r.bad || x->nt < 1 || x->npc < 1 || x->nt > 64 || x->npc > 64) { pjo_mech_free(m); return PJO_EFORMAT; }
            for (int c = 0; c < 4; ++c) x->cheb_rng[c] = rdd(&r);
            x->eta = malloc((size_t)x->nt * x->npc * sizeof(double));
            if (!x->eta) { pjo_mech_free(m); return PJO_ENOMEM; }
            for (int c = 0; c < x->nt * x->npc; ++c) x->eta[c] = rdd(&r);
        }
        if (r.bad) { pjo_mech_free(m); return PJO_EFORMAT; }
        /* net stoichiometric coefficients nu_ki = nu''_ki - nu'_ki */
        x->nnet = 0;
        for (int pass = 0; pass < 2; ++pass) {
            int n = pass ? x->np : x->nr;
            const int *sp = pass ? x->psp : x->rsp, *nu = pass ? x->pnu : x->rnu;
            for (int s = 0; s < n; ++s) {
                int v = pass ? nu[s] : -nu[s], found = 0;
                for (int t = 0; t < x->nnet; ++t)
                    if (x->netsp[t] == sp[s]) { x->netnu[t] += v; found = 1; }
                if (!found) { x->netsp[x->nnet] = sp[s]; x->netnu[x->nnet] = v; x->nnet++; }
            }
        }
        int w = 0;
        for (int t = 0; t < x->nnet; ++t)
            if (x->netnu[t] != 0) { x->netsp[w] = x->netsp[t]; x->netnu[w] = x->netnu[t]; ++w; }
        x->nnet = w;
    }
    if (r.p != r.end) { pjo_mech_free(m); return PJO_EFORMAT; }
    *out = m;
    return PJO_OK;
}

int pjo_mech_info(const pjo_mech *m, int *ns, int *nr, int *ne)
{
    if (!m) return PJO_EINVAL;
    if (ns) *ns = m->ns;
    if (nr) *nr = m->nr;
    if (ne) *ne = m->ne;
    return PJO_OK;
}

static int g_threads = 0;
void pjo_set_threads(int n) { g_threads = n; }
int pjo_max_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------------------
 * Source terms over a batch. */

int pjo_eval_dydt(const pjo_mech *m, int64_t n, const double *T, const double *P, const double *Y, int64_t ldy,
                  double *dydt, int64_t ldd)
{
    if (!m || n < 0 || ldy < m->ns || ldd < m->ns + 1) return PJO_EINVAL;
    if (n == 0) return PJO_OK;
    if (!T || !P || !Y || !dydt) return PJO_EINVAL;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(pjo_max_threads())
    for (int64_t s = 0; s < n; ++s) {
        double *wk = malloc((6 * (size_t)m->ns + 2 * (size_t)m->nr + 8) * sizeof(double));
        if (!wk) { err = 1; continue; }
        source_terms_d(m, T[s], P[s], Y + s * ldy, dydt + s * ldd, NULL, wk);
        free(wk);
    }
    return err ? PJO_ENOMEM : PJO_OK;
}

/* Per-reaction values for one state (for the oracle's own pins): kf, kr, c, R_f, R_r, q. */
int pjo_reaction_rates(const pjo_mech *m, double T, double P, const double *Y,
                       double *kf, double *kr, double *c, double *Rf, double *Rr, double *q)
{
    if (!m || !Y) return PJO_EINVAL;
    int N = m->ns;
    double *C = malloc(2 * N * sizeof(double));
    if (!C) return PJO_ENOMEM;
    double *B = C + N;
    double sYW = 0.0;
    for (int k = 0; k < N; ++k) sYW += Y[k] / m->W[k];
    double rho = P / (sYW * PJO_R * T);
    for (int k = 0; k < N; ++k) { C[k] = rho * Y[k] / m->W[k]; B[k] = Bk_d(m, k, T); }
    for (int i = 0; i < m->nr; ++i) {
        double a, b, cc, d, e;
        rxn_rates_d(m, i, T, P, C, B, &a, &b, &cc, &d, &e);
        if (kf) kf[i] = a;
        if (kr) kr[i] = b;
        if (c) c[i] = cc;
        if (Rf) Rf[i] = d;
        if (Rr) Rr[i] = e;
        if (q) q[i] = cc * (d - e);
    }
    free(C);
    return PJO_OK;
}

/* Per-species thermodynamic values at T: cp/R, H/(R T), S/R, B_k (Eqs. e:cpk, e:hk, e:sk). */
int pjo_species_thermo(const pjo_mech *m, double T, double *cpR, double *HRT, double *SR, double *B)
{
    if (!m) return PJO_EINVAL;
    for (int k = 0; k < m->ns; ++k) {
        double a, b, c;
        nasa7_d(m, k, T, &a, &b, &c);
        if (cpR) cpR[k] = a;
        if (HRT) HRT[k] = b;
        if (SR) SR[k] = c;
        if (B) B[k] = Bk_d(m, k, T);
    }
    return PJO_OK;
}

/* ---------------------------------------------------------------------------------------------
 * Analytical Jacobian, Section 3.1, one state. */

typedef struct { double s, c; } csum;
static void cs_add(csum *a, double x) { acc_d(&a->s, &a->c, x); }
static double cs_val(const csum *a) { return a->s + a->c; }

/* Troe F and its partial derivatives dF/dFcent, dF/dP_r and Fcent, dFcent/dT (Section 3.1); dFdlnPr
 * receives P_r dF/dP_r, which stays finite at P_r = 0. */
static void troe_parts(const pjo_rxn *r, double T, double Pr, double *F, double *dFdT_Pr, double *dFdPr,
                       double *dFdlnPr)
{
    double a = r->fp[0], T3 = r->fp[1], T1 = r->fp[2], T2 = r->fp[3];
    double Fc = (1.0 - a) * exp(-T / T3) + a * exp(-T / T1) + (r->has_T2 ? exp(-T2 / T) : 0.0);
    double dFc = -(1.0 - a) / T3 * exp(-T / T3) - a / T1 * exp(-T / T1) + (r->has_T2 ? T2 / (T * T) * exp(-T2 / T) : 0.0);
    double Prc = Pr < 1e-300 ? 1e-300 : Pr;
    double lFc = log10(Fc), lPr = log10(Prc);
    double At = lPr - 0.67 * lFc - 0.4;
    double Bt = 0.806 - 1.1762 * lFc - 0.14 * lPr;
    double g = 1.0 + (At / Bt) * (At / Bt);
    double Fv = pow(Fc, 1.0 / g);
    double dAdFc = -0.67 / (Fc * M_LN10), dBdFc = -1.1762 / (Fc * M_LN10);
    double dAdPr = 1.0 / (Pr * M_LN10), dBdPr = -0.14 / (Pr * M_LN10);
    double dFdFc = Fv * (1.0 / (Fc * g) - log(Fc) * 2.0 * At / (Bt * Bt * Bt) * (dAdFc * Bt - At * dBdFc) / (g * g));
    *dFdPr = -Fv * log(Fc) * 2.0 * At / (Bt * Bt * Bt) * (dAdPr * Bt - At * dBdPr) / (g * g);
    *dFdlnPr = -Fv * log(Fc) * 2.0 * At / (Bt * Bt * Bt) * (1.0 / M_LN10 * Bt - At * (-0.14 / M_LN10)) / (g * g);
    if (Pr < 1e-300) *dFdPr = *dFdlnPr = 0.0;   /* F is constant below the clamp */
    *F = Fv;
    *dFdT_Pr = dFdFc * dFc;   /* explicit temperature dependence at fixed P_r */
}

/* SRI F, its explicit T-derivative at fixed P_r, dF/dP_r and P_r dF/dP_r (Section 3.1). */
static void sri_parts(const pjo_rxn *r, double T, double Pr, double *F, double *dFdT_Pr, double *dFdPr,
                      double *dFdlnPr)
{
    double a = r->fp[0], b = r->fp[1], c = r->fp[2], d = r->fp[3], e = r->fp[4];
    double Prc = Pr < 1e-300 ? 1e-300 : Pr;
    double lPr = log10(Prc);
    double X = 1.0 / (1.0 + lPr * lPr);
    double base = a * exp(-b / T) + exp(-T / c);
    double Fv = d * pow(T, e) * pow(base, X);
    double dXdPr = -X * X * 2.0 * lPr / (Pr * M_LN10);
    *F = Fv;
    *dFdT_Pr = Fv * (e / T + X * (a * b / (T * T) * exp(-b / T) - exp(-T / c) / c) / base);
    *dFdPr = Fv * dXdPr * log(base);
    *dFdlnPr = Fv * (-X * X * 2.0 * lPr / M_LN10) * log(base);
    if (Pr < 1e-300) *dFdPr = *dFdlnPr = 0.0;   /* F is constant below the clamp */
}

/* Chebyshev polynomial of the second kind U_n(x) by its recurrence (U_0 = 1, U_1 = 2x). */
static double chebU(int n, double x)
{
    double u0 = 1.0, u1 = 2.0 * x;
    if (n == 0) return u0;
    for (int k = 2; k <= n; ++k) { double u2 = 2.0 * x * u1 - u0; u0 = u1; u1 = u2; }
    return u1;
}

/* dk_f/dT for reaction i (Eq. e:dkfdT and the PLOG / Chebyshev forms of Section 3.1). */
static double dkf_dT(const pjo_rxn *r, double T, double P, double kf)
{
    switch (r->kind) {
    case PJO_ELEM:
    case PJO_THIRD:
        return kf / T * (r->beta + r->Ta / T);
    case PJO_FALLOFF:
        return kf / T * (r->kinf[1] + r->kinf[2] / T);
    case PJO_CHEM:
        return kf / T * (r->k0[1] + r->k0[2] / T);
    case PJO_PLOG: {
        const double *t = r->plog;
        int n = r->nplog;
        if (P <= t[0]) return kf / T * (t[2] + t[3] / T);
        if (P >= t[4 * (n - 1)]) return kf / T * (t[4 * (n - 1) + 2] + t[4 * (n - 1) + 3] / T);
        int i = 0;
        while (!(t[4 * i] <= P && P < t[4 * (i + 1)])) ++i;
        const double *a = &t[4 * i], *b = &t[4 * (i + 1)];
        double fr = (log(P) - log(a[0])) / (log(b[0]) - log(a[0]));
        return kf / T * (a[2] + a[3] / T + (b[2] - a[2] + (b[3] - a[3]) / T) * fr);
    }
    case PJO_CHEB: {
        double Tmin = r->cheb_rng[0], Tmax = r->cheb_rng[1], Pmin = r->cheb_rng[2], Pmax = r->cheb_rng[3];
        double Tt = (2.0 / T - 1.0 / Tmin - 1.0 / Tmax) / (1.0 / Tmax - 1.0 / Tmin);
        double pt = (2.0 * log10(P) - log10(Pmin) - log10(Pmax)) / (log10(Pmax) - log10(Pmin));
        double dTt = -2.0 / (T * T) / (1.0 / Tmax - 1.0 / Tmin);
        double s = 0.0;
        for (int i = 1; i < r->nt; ++i)   /* d/dx T_i(x) = i U_{i-1}(x) */
            for (int j = 0; j < r->npc; ++j) s += r->eta[i * r->npc + j] * i * chebU(i - 1, Tt) * chebT_d(j, pt);
        return M_LN10 * kf * s * dTt;
    }
    }
    return 0.0;
}

static int jac_one(const pjo_mech *m, double T, double P, const double *Y,
                   double *J, double *Jsc, double *f, double *fsc)
{
    const int N = m->ns, R = m->nr, Nj = N - 1, L = N - 1; /* L: index of the last species */
    size_t need = (size_t)N * 12 + (size_t)R * 8 + 2 * (size_t)R * Nj + 3 * (size_t)N * N;
    double *buf = calloc(need, sizeof(double));
    if (!buf) return PJO_ENOMEM;
    double *C = buf, *cpk = C + N, *hk = cpk + N, *dcpk = hk + N, *B = dcpk + N, *dB = B + N, *Dl = dB + N;
    double *om = Dl + N, *omabs = om + N;
    double *fk = omabs + N, *fkabs = fk + N, *spare = fkabs + N;
    double *kfv = spare + N, *krv = kfv + R, *cv = krv + R, *Rfv = cv + R, *Rrv = Rfv + R;
    double *dqT = Rrv + R, *dqTabs = dqT + R, *Rabs = dqTabs + R;
    double *dqY = Rabs + R, *dqYabs = dqY + (size_t)R * Nj;
    double *Ssum = dqYabs + (size_t)R * Nj, *Scmp = Ssum + (size_t)N * N, *Sabs = Scmp + (size_t)N * N;
    (void)spare;

    /* state: W, rho, [X_k] (Section 2.1) */
    csum sYW = {0, 0};
    for (int k = 0; k < N; ++k) cs_add(&sYW, Y[k] / m->W[k]);
    const double Wm = 1.0 / cs_val(&sYW);
    const double rho = P * Wm / (PJO_R * T);
    for (int k = 0; k < N; ++k) C[k] = rho * Y[k] / m->W[k];
    /* thermo (Section 2.2) and the derivatives of Section 3.1 */
    csum scp = {0, 0}, sdcp = {0, 0};
    for (int k = 0; k < N; ++k) {
        double cpR, HRT, SR;
        nasa7_d(m, k, T, &cpR, &HRT, &SR);
        const double *a = (T < m->Tmid[k]) ? &m->alo[7 * k] : &m->ahi[7 * k];
        cpk[k] = cpR * PJO_R / m->W[k];
        hk[k] = HRT * PJO_R * T / m->W[k];
        dcpk[k] = PJO_R / m->W[k] * (a[1] + T * (2.0 * a[2] + T * (3.0 * a[3] + 4.0 * a[4] * T)));
        B[k] = Bk_d(m, k, T);
        dB[k] = (a[0] - 1.0 + a[5] / T) / T + a[1] / 2.0 + T * (a[2] / 3.0 + T * (a[3] / 4.0 + a[4] / 5.0 * T));
        cs_add(&scp, Y[k] * cpk[k]);
        cs_add(&sdcp, Y[k] * dcpk[k]);        /* Eq. E:dcpdT */
    }
    const double cp = cs_val(&scp), dcpdT = cs_val(&sdcp);
    for (int j = 0; j < Nj; ++j) Dl[j] = 1.0 / m->W[j] - 1.0 / m->W[L];
    const double drhodT = -rho / T;

    /* per reaction: rates and the derivatives of q_i = c_i R_i */
    for (int i = 0; i < R; ++i) {
        const pjo_rxn *r = &m->rx[i];
        double kf, kr, c, Rf, Rr;
        rxn_rates_d(m, i, T, P, C, B, &kf, &kr, &c, &Rf, &Rr);
        kfv[i] = kf; krv[i] = kr; cv[i] = c; Rfv[i] = Rf; Rrv[i] = Rr;
        const double Rn = Rf - Rr;
        Rabs[i] = fabs(Rf) + fabs(Rr);
        double nf = 0.0, nb = 0.0;
        for (int s = 0; s < r->nr; ++s) nf += r->rnu[s];
        for (int s = 0; s < r->np; ++s) nb += r->pnu[s];
        /* rate coefficient temperature derivatives */
        const double dkf = dkf_dT(r, T, P, kf);
        double dkr = 0.0;
        if (r->rev == PJO_REV_KC) {
            /* Eq. e:dkrdT_general with dK_c/dT = K_c sum_k nu_k dB_k/dT */
            double sB = 0.0, sdB = 0.0;
            int dn = 0;
            for (int s = 0; s < r->np; ++s) { sB += r->pnu[s] * B[r->psp[s]]; sdB += r->pnu[s] * dB[r->psp[s]]; dn += r->pnu[s]; }
            for (int s = 0; s < r->nr; ++s) { sB -= r->rnu[s] * B[r->rsp[s]]; sdB -= r->rnu[s] * dB[r->rsp[s]]; dn -= r->rnu[s]; }
            double Kc = pow(PJO_PATM / PJO_R, (double)dn) * exp(sB);
            double dKc = Kc * sdB;
            dkr = (dkf * Kc - dKc * kf) / (Kc * Kc);
        } else if (r->rev == PJO_REV_EXPLICIT) {
            dkr = kr / T * (r->betar + r->Tar / T);
        }
        /* concentration products and their T derivative */
        double Pf = 1.0, Pb = 1.0;
        for (int s = 0; s < r->nr; ++s) Pf *= ipow_d(C[r->rsp[s]], r->rnu[s]);
        for (int s = 0; s < r->np; ++s) Pb *= ipow_d(C[r->psp[s]], r->pnu[s]);
        const double dPfdT = -Pf / T * nf, dPbdT = -Pb / T * nb;
        const double dRfdT = dkf * Pf + kf * dPfdT;            /* Eq. E:dRfdT-orig */
        const double dRrdT = dkr * Pb + kr * dPbdT;
        const double dRdT = dRfdT - dRrdT;
        const double dRdTabs = fabs(dkf * Pf) + fabs(kf * dPfdT) + fabs(dkr * Pb) + fabs(kr * dPbdT);

        /* pressure modifier derivatives */
        double dcdT = 0.0, dcdTabs = 0.0;
        double Pr = 0.0, ratio = 0.0, Fv = 1.0, dFdPr = 0.0, dFdlnPr = 0.0, M = 0.0;
        if (r->kind == PJO_THIRD) {
            dcdT = -c / T;
            dcdTabs = fabs(dcdT);
        } else if (r->kind == PJO_FALLOFF || r->kind == PJO_CHEM) {
            double k0 = arrhenius_d(r->k0[0], r->k0[1], r->k0[2], T);
            double ki = arrhenius_d(r->kinf[0], r->kinf[1], r->kinf[2], T);
            M = third_body_d(m, r, C);
            ratio = k0 / ki;
            Pr = ratio * M;
            /* Eq. E:dPridT */
            double dPrdT = Pr / T * (r->k0[1] - r->kinf[1] + (r->k0[2] - r->kinf[2]) / T - 1.0);
            double dFdT = 0.0, dFdT_Pr = 0.0;
            if (r->ftype == PJO_TROE) troe_parts(r, T, Pr, &Fv, &dFdT_Pr, &dFdPr, &dFdlnPr);
            else if (r->ftype == PJO_SRI) sri_parts(r, T, Pr, &Fv, &dFdT_Pr, &dFdPr, &dFdlnPr);
            if (Pr < 1e-300 && r->kind == PJO_FALLOFF) {
                /* P_r = 0 (a single third-body species that is absent): c = 0 and P_r ~ [M], so the
                 * limit of Eq. dCidT is 0; the 1/P_r form would be 0 * inf */
                dcdT = 0.0;
                dcdTabs = 0.0;
            } else {
                dFdT = dFdT_Pr + dFdPr * dPrdT;
                if (r->kind == PJO_FALLOFF) dcdT = c * (1.0 / (Pr * (1.0 + Pr)) * dPrdT + dFdT / Fv);
                else                        dcdT = c * (-1.0 / (1.0 + Pr) * dPrdT + dFdT / Fv);
                /* the scale counts the terms of the kind's own form (the falloff one alone has 1/P_r) */
                const double tPr = r->kind == PJO_FALLOFF ? fabs(dPrdT / (Pr * (1.0 + Pr))) : fabs(dPrdT / (1.0 + Pr));
                dcdTabs = fabs(c) * (tPr + fabs(dFdT_Pr / Fv) + fabs(dFdPr * dPrdT / Fv));
            }
        }
        dqT[i] = dcdT * Rn + c * dRdT;
        dqTabs[i] = dcdTabs * Rabs[i] + fabs(c) * dRdTabs;

        /* species-mass-fraction derivatives, j = 0..N-2 (column j+1) */
        for (int j = 0; j < Nj; ++j) {
            /* d(prod [X]^nu')/dY_j, Section 3.1 */
            double dPf = 0.0, dPfa = 0.0, dPb = 0.0, dPba = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                int n = pass ? r->np : r->nr;
                const int *sp = pass ? r->psp : r->rsp, *nu = pass ? r->pnu : r->rnu;
                double acc = 0.0, acca = 0.0;
                for (int s = 0; s < n; ++s) {
                    int k = sp[s];
                    double others = 1.0;
                    for (int t = 0; t < n; ++t) if (t != s) others *= ipow_d(C[sp[t]], nu[t]);
                    double t1 = -ipow_d(C[k], nu[s]) * Wm * Dl[j];
                    double dl = (k == j ? 1.0 : 0.0) - (k == L ? 1.0 : 0.0);
                    double t2 = dl * rho / m->W[k] * ipow_d(C[k], nu[s] - 1);
                    acc += nu[s] * (t1 + t2) * others;
                    acca += nu[s] * (fabs(t1) + fabs(t2)) * fabs(others);
                }
                if (pass) { dPb = acc; dPba = acca; } else { dPf = acc; dPfa = acca; }
            }
            double dRdY = kf * dPf - kr * dPb;
            double dRdYabs = fabs(kf) * dPfa + fabs(kr) * dPba;
            double dcdY = 0.0, dcdYabs = 0.0;
            if (r->kind == PJO_THIRD) {
                if (r->tb_mode == PJO_TB_MIX) {
                    double t2 = rho * (r->alpha[j] / m->W[j] - r->alpha[L] / m->W[L]);
                    dcdY = -Wm * c * Dl[j] + t2;
                    dcdYabs = fabs(Wm * c * Dl[j]) + rho * (fabs(r->alpha[j]) / m->W[j] + fabs(r->alpha[L]) / m->W[L]);
                } else {
                    int ms = r->tb_sp;
                    double dl = (ms == j ? 1.0 : 0.0) - (ms == L ? 1.0 : 0.0);
                    dcdY = -C[ms] * Wm * Dl[j] + dl * rho / m->W[ms];
                    dcdYabs = fabs(C[ms] * Wm * Dl[j]) + fabs(dl) * rho / m->W[ms];
                }
            } else if (r->kind == PJO_FALLOFF || r->kind == PJO_CHEM) {
                double dPrdY, dPrdYabs;
                if (r->tb_mode == PJO_TB_MIX) {   /* Eq. E:dPridY, mixture */
                    double t2 = ratio * rho * (r->alpha[j] / m->W[j] - r->alpha[L] / m->W[L]);
                    dPrdY = -Pr * Wm * Dl[j] + t2;
                    dPrdYabs = fabs(Pr * Wm * Dl[j]) + ratio * rho * (fabs(r->alpha[j]) / m->W[j] + fabs(r->alpha[L]) / m->W[L]);
                } else {                          /* Eq. E:dPridY, species m */
                    int ms = r->tb_sp;
                    double dl = (ms == j ? 1.0 : 0.0) - (ms == L ? 1.0 : 0.0);
                    dPrdY = -Pr * Wm * Dl[j] + ratio * rho / m->W[ms] * dl;
                    dPrdYabs = fabs(Pr * Wm * Dl[j]) + ratio * rho / m->W[ms] * fabs(dl);
                }
                double dFdY = dFdPr * dPrdY;
                if (Pr < 1e-300 && r->kind == PJO_FALLOFF) {
                    /* the limit of Eq. dCidY_falloff at P_r = 0, from c / P_r = F / (1 + P_r) and
                     * c dF/dP_r / F = P_r dF/dP_r / (1 + P_r): dc/dY = (F + P_r dF/dP_r) dP_r/dY */
                    dcdY = (Fv + dFdlnPr) * dPrdY;
                    dcdYabs = (fabs(Fv) + fabs(dFdlnPr)) * dPrdYabs;
                } else {
                    if (r->kind == PJO_FALLOFF) dcdY = c * (1.0 / (Pr * (1.0 + Pr)) * dPrdY + dFdY / Fv);   /* Eq. dCidY_falloff */
                    else                        dcdY = c * (-1.0 / (1.0 + Pr) * dPrdY + dFdY / Fv);         /* Eq. dCidY_chem */
                    const double tPr = r->kind == PJO_FALLOFF ? fabs(1.0 / (Pr * (1.0 + Pr))) : 1.0 / (1.0 + Pr);
                    dcdYabs = fabs(c) * (tPr + fabs(dFdPr / Fv)) * dPrdYabs;
                }
            }
            dqY[(size_t)i * Nj + j] = dcdY * Rn + c * dRdY;
            dqYabs[(size_t)i * Nj + j] = dcdYabs * Rabs[i] + fabs(c) * dRdYabs;
        }
        (void)M;
    }

    /* omega_k = sum_i nu_ki q_i */
    for (int k = 0; k < N; ++k) { om[k] = 0.0; omabs[k] = 0.0; }
    {
        double *omc = calloc(N, sizeof(double));
        if (!omc) { free(buf); return PJO_ENOMEM; }
        for (int i = 0; i < R; ++i) {
            const pjo_rxn *r = &m->rx[i];
            double q = cv[i] * (Rfv[i] - Rrv[i]);
            for (int s = 0; s < r->nnet; ++s) {
                int k = r->netsp[s];
                acc_d(&om[k], &omc[k], r->netnu[s] * q);
                omabs[k] += fabs((double)r->netnu[s]) * fabs(cv[i]) * Rabs[i];
            }
        }
        for (int k = 0; k < N; ++k) om[k] += omc[k];
        free(omc);
    }
    for (int k = 0; k < N; ++k) {
        fk[k] = m->W[k] * om[k] / rho;
        fkabs[k] = m->W[k] * omabs[k] / rho;
    }

    /* species rows k = 1..N (Eq. e:jac_spec): sums over reactions, column 0 = T */
    for (size_t e = 0; e < (size_t)N * N; ++e) { Ssum[e] = 0.0; Scmp[e] = 0.0; Sabs[e] = 0.0; }
    for (int i = 0; i < R; ++i) {
        const pjo_rxn *r = &m->rx[i];
        for (int s = 0; s < r->nnet; ++s) {
            int k = r->netsp[s];
            double nu = r->netnu[s];
            double *row = Ssum + (size_t)k * N, *cmp = Scmp + (size_t)k * N, *ab = Sabs + (size_t)k * N;
            acc_d(&row[0], &cmp[0], nu * dqT[i]);
            ab[0] += fabs(nu) * dqTabs[i];
            for (int j = 0; j < Nj; ++j) {
                acc_d(&row[1 + j], &cmp[1 + j], nu * dqY[(size_t)i * Nj + j]);
                ab[1 + j] += fabs(nu) * dqYabs[(size_t)i * Nj + j];
            }
        }
    }
    const int ld = N + 1;
    for (int k = 0; k < N; ++k) {
        double *row = Ssum + (size_t)k * N, *cmp = Scmp + (size_t)k * N, *ab = Sabs + (size_t)k * N;
        double pre = m->W[k] / rho;
        /* J_{k+1,1} = W_k/rho (domega_k/dT - omega_k/rho drho/dT) */
        acc_d(&row[0], &cmp[0], -om[k] / rho * drhodT);
        J[(size_t)(1 + k) * ld + 0] = pre * (row[0] + cmp[0]);
        if (Jsc) Jsc[(size_t)(1 + k) * ld + 0] = pre * (ab[0] + omabs[k] / T);
        for (int j = 0; j < Nj; ++j) {
            /* J_{k+1,j+1} = W_k/rho (domega_k/dY_j - omega_k/rho drho/dY_j), drho/dY_j = -rho W Delta_j */
            acc_d(&row[1 + j], &cmp[1 + j], om[k] * Wm * Dl[j]);
            J[(size_t)(1 + k) * ld + 1 + j] = pre * (row[1 + j] + cmp[1 + j]);
            if (Jsc) Jsc[(size_t)(1 + k) * ld + 1 + j] = pre * (ab[1 + j] + omabs[k] * Wm * fabs(Dl[j]));
        }
        J[(size_t)(1 + k) * ld + N] = 0.0;
        if (Jsc) Jsc[(size_t)(1 + k) * ld + N] = 0.0;
    }

    /* energy row (Eq. e:jac_dt) */
    csum hwo = {0, 0};
    double hwoabs = 0.0;
    for (int k = 0; k < N; ++k) {
        cs_add(&hwo, hk[k] * m->W[k] * om[k]);
        hwoabs += fabs(hk[k]) * m->W[k] * omabs[k];
    }
    const double HWO = cs_val(&hwo);
    {
        csum s = {0, 0};
        double sa = 0.0;
        for (int k = 0; k < N; ++k) {
            cs_add(&s, (cpk[k] - hk[k] / cp * dcpdT) * fk[k]);
            cs_add(&s, hk[k] * J[(size_t)(1 + k) * ld + 0]);
            sa += (fabs(cpk[k]) + fabs(hk[k] / cp * dcpdT)) * fkabs[k] +
                  fabs(hk[k]) * (Jsc ? Jsc[(size_t)(1 + k) * ld + 0] : 0.0);
        }
        J[0] = -cs_val(&s) / cp;
        if (Jsc) Jsc[0] = sa / cp;
    }
    for (int j = 0; j < Nj; ++j) {
        csum s = {0, 0};
        double sa = 0.0;
        cs_add(&s, -(cpk[j] - cpk[L]) / (rho * cp) * HWO);
        sa += fabs(cpk[j] - cpk[L]) / (rho * cp) * hwoabs;
        for (int k = 0; k < N; ++k) {
            cs_add(&s, hk[k] * J[(size_t)(1 + k) * ld + 1 + j]);
            sa += fabs(hk[k]) * (Jsc ? Jsc[(size_t)(1 + k) * ld + 1 + j] : 0.0);
        }
        J[1 + j] = -cs_val(&s) / cp;
        if (Jsc) Jsc[1 + j] = sa / cp;
    }
    J[N] = 0.0;
    if (Jsc) Jsc[N] = 0.0;

    if (f) {
        f[0] = -HWO / (rho * cp);
        for (int k = 0; k < N; ++k) f[1 + k] = fk[k];
    }
    if (fsc) {
        fsc[0] = hwoabs / (rho * cp);
        for (int k = 0; k < N; ++k) fsc[1 + k] = fkabs[k];
    }
    free(buf);
    return PJO_OK;
}

int pjo_eval_jacobian(const pjo_mech *m, int64_t n, const double *T, const double *P, const double *Y, int64_t ldy,
                      double *jac, int64_t ldj, double *jac_scale, double *dydt, int64_t ldd, double *dydt_scale)
{
    if (!m || n < 0 || ldy < m->ns) return PJO_EINVAL;
    int64_t nn = (int64_t)(m->ns + 1) * (m->ns + 1);
    if (ldj < nn) return PJO_EINVAL;
    if ((dydt || dydt_scale) && ldd < m->ns + 1) return PJO_EINVAL;
    if (n == 0) return PJO_OK;
    if (!T || !P || !Y || !jac) return PJO_EINVAL;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(pjo_max_threads())
    for (int64_t s = 0; s < n; ++s) {
        int rc = jac_one(m, T[s], P[s], Y + s * ldy, jac + s * ldj, jac_scale ? jac_scale + s * ldj : NULL,
                         dydt ? dydt + s * ldd : NULL, dydt_scale ? dydt_scale + s * ldd : NULL);
        if (rc) err = rc;
    }
    return err;
}

/* First-order forward-difference Jacobian: the finite-difference comparison of the paper's
 * performance section (a first-order forward difference adapted from CVODE). Column 0 moves T,
 * column j (1..N-1) moves Y_j by +h_j and Y_N by -h_j (the directions of the analytical columns),
 * column N is zero. Increment h_c = 2^-26 max(|y_c|, a_c) with a_0 = 1 K and a_c = 1e-10 for mass
 * fractions: CVODE's relative increment sqrt(unit roundoff) |y_c|, with a fixed floor in place of
 * its error-weight term (which needs an integrator's tolerances and step size). 2^-26 is exactly
 * sqrt(DBL_EPSILON). J_kc = (f_k(y + h_c d_c) - f_k(y)) / h_c. With jac_scale, each entry also
 * gets (S_k(y + h_c d_c) + S_k(y)) / h_c, S the source-term scale (sum of the absolute values of
 * the terms of f_k): a bound on how far rounding in f can move the entry. */
static double fd_increment(int c, double T, const double *Y)
{
    const double y = c == 0 ? T : Y[c - 1], a = c == 0 ? 1.0 : 1e-10;
    return 0x1p-26 * fmax(fabs(y), a);
}

int pjo_jacobian_fd(const pjo_mech *m, int64_t n, const double *T, const double *P, const double *Y, int64_t ldy,
                    double *jac, int64_t ldj, double *jac_scale)
{
    if (!m || n < 0 || ldy < m->ns) return PJO_EINVAL;
    const int N = m->ns;
    if (ldj < (int64_t)(N + 1) * (N + 1)) return PJO_EINVAL;
    if (n == 0) return PJO_OK;
    if (!T || !P || !Y || !jac) return PJO_EINVAL;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(pjo_max_threads())
    for (int64_t s = 0; s < n; ++s) {
        /* f and its per-entry term scale come from the Jacobian routine (its J is discarded) */
        double *buf = malloc(((size_t)N + 4 * ((size_t)N + 1) + (size_t)(N + 1) * (N + 1)) * sizeof(double));
        if (!buf) { err = 1; continue; }
        double *Yp = buf, *f0 = Yp + N, *s0 = f0 + N + 1, *f1 = s0 + N + 1, *s1 = f1 + N + 1, *Jt = s1 + N + 1;
        const double *Ys = Y + s * ldy;
        double *Jo = jac + s * ldj, *Jso = jac_scale ? jac_scale + s * ldj : NULL;
        int rc = jac_one(m, T[s], P[s], Ys, Jt, NULL, f0, s0);
        for (int col = 0; col < N + 1; ++col) {
            if (col == N) {
                for (int row = 0; row < N + 1; ++row) {
                    Jo[(size_t)row * (N + 1) + col] = 0.0;
                    if (Jso) Jso[(size_t)row * (N + 1) + col] = 0.0;
                }
                continue;
            }
            const double h = fd_increment(col, T[s], Ys);
            double Tp = T[s];
            for (int k = 0; k < N; ++k) Yp[k] = Ys[k];
            if (col == 0) Tp = T[s] + h;
            else { Yp[col - 1] = Ys[col - 1] + h; Yp[N - 1] = Ys[N - 1] - h; }
            rc |= jac_one(m, Tp, P[s], Yp, Jt, NULL, f1, s1);
            for (int row = 0; row < N + 1; ++row) {
                Jo[(size_t)row * (N + 1) + col] = (f1[row] - f0[row]) / h;
                if (Jso) Jso[(size_t)row * (N + 1) + col] = (s1[row] + s0[row]) / h;
            }
        }
        free(buf);
        if (rc) err = 1;
    }
    return err ? PJO_ENOMEM : PJO_OK;
}

/* ---------------------------------------------------------------------------------------------
 * Constant volume (Section 3.3): source terms of the state (T, rho, Y), and their Jacobian by the
 * plain definition, d f / d y along the analytical columns (T; Y_j with Y_N = 1 - sum of the
 * others; column N zero), evaluated by complex-step differentiation of the source terms. A species
 * column is the difference of two one-species directional derivatives, d f / d Y_j - d f / d Y_N
 * (the same linear map as one step along Y_j - Y_N); the optional per-entry scale bounds the
 * rounding of an entry: (W_k/rho) sum_i |nu_ki| (|d(c R_f)_i| + |d(c R_r)_i|) summed over the
 * column's directions (T alone, or Y_j and Y_N separately, so that an entry formed from two large
 * and nearly equal contributions, e.g. through 1/W_j - 1/W_N for W_j close to W_N, carries their
 * size), and for the energy row the same sums weighted by |u_k W_k| plus |du_k W_k omega_k| and
 * |f_0 dc_v|, over rho c_v. */
int pjo_eval_dydt_cv(const pjo_mech *m, int64_t n, const double *T, const double *rho, const double *Y, int64_t ldy,
                     double *dydt, int64_t ldd, double *dydt_scale)
{
    if (!m || n < 0 || ldy < m->ns || ldd < m->ns + 1) return PJO_EINVAL;
    if (n == 0) return PJO_OK;
    if (!T || !rho || !Y || !dydt) return PJO_EINVAL;
    const int N = m->ns, R = m->nr;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(pjo_max_threads())
    for (int64_t s = 0; s < n; ++s) {
        double *wk = malloc((6 * (size_t)N + 2 * (size_t)R + 8 + 2 * (size_t)R + N) * sizeof(double));
        if (!wk) { err = 1; continue; }
        double *qf = wk + 6 * (size_t)N + 2 * (size_t)R + 8, *qr = qf + R, *sk = qr + R;
        const double *Ys = Y + s * ldy;
        source_terms_cv_d(m, T[s], rho[s], Ys, dydt + s * ldd, qf, qr, wk);
        if (dydt_scale) {
            /* per entry: the sum of the absolute values of its terms, sum_i |nu_ki| (|c R_f| + |c R_r|)
             * for species k (times W_k / rho), and sum_k |u_k W_k| of those over rho c_v for T;
             * c_v,k and u_k are left in wk by the source terms */
            const double *cvk = wk + 2 * (size_t)N, *uk = wk + 3 * (size_t)N;
            double cv = 0.0;
            for (int k = 0; k < N; ++k) { sk[k] = 0.0; cv += Ys[k] * cvk[k]; }
            for (int i = 0; i < R; ++i) {
                const pjo_rxn *r = &m->rx[i];
                for (int q = 0; q < r->nnet; ++q) sk[r->netsp[q]] += fabs(r->netnu[q]) * (fabs(qf[i]) + fabs(qr[i]));
            }
            double *sc = dydt_scale + s * ldd, e0 = 0.0;
            for (int k = 0; k < N; ++k) {
                sc[1 + k] = m->W[k] / rho[s] * sk[k];
                e0 += fabs(uk[k] * m->W[k]) * sk[k];
            }
            sc[0] = e0 / (rho[s] * cv);
        }
        free(wk);
    }
    return err ? PJO_ENOMEM : PJO_OK;
}

int pjo_jacobian_cv(const pjo_mech *m, int64_t n, const double *T, const double *rho, const double *Y, int64_t ldy,
                    double *jac, int64_t ldj, double *jac_scale)
{
    if (!m || n < 0 || ldy < m->ns) return PJO_EINVAL;
    const int N = m->ns, R = m->nr;
    if (ldj < (int64_t)(N + 1) * (N + 1)) return PJO_EINVAL;
    if (n == 0) return PJO_OK;
    if (!T || !rho || !Y || !jac) return PJO_EINVAL;
    const double h = 1e-30;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(pjo_max_threads())
    for (int64_t s = 0; s < n; ++s) {
        const size_t nwk = 6 * (size_t)N + 2 * (size_t)R + 8;
        size_t nz = (size_t)N + (N + 1) + 2 * (size_t)R + nwk;
        /* f, qf, qr, wk; c_v,k, u_k, dc_v,k/dT; the Y_N direction: d f, |d(cR_f)|, |d(cR_r)|; sk */
        size_t nd = (size_t)(N + 1) + 2 * (size_t)R + nwk + 3 * (size_t)N + (size_t)(N + 1) + 2 * (size_t)R + N;
        double complex *Yz = malloc(nz * sizeof(double complex));
        double *bd = malloc(nd * sizeof(double));
        if (!Yz || !bd) { free(Yz); free(bd); err = 1; continue; }
        double complex *fz = Yz + N, *qfz = fz + N + 1, *qrz = qfz + R, *wkz = qrz + R;
        double *f = bd, *qf = f + N + 1, *qr = qf + R, *wk = qr + R, *cvk = wk + nwk, *uk = cvk + N, *dcvk = uk + N;
        double *dfN = dcvk + N, *aqfN = dfN + N + 1, *aqrN = aqfN + R, *sk = aqrN + R;
        const double *Ys = Y + s * ldy;
        const double r0 = rho[s];
        double *Jo = jac + s * ldj, *Jso = jac_scale ? jac_scale + s * ldj : NULL;
        source_terms_cv_d(m, T[s], r0, Ys, f, qf, qr, wk);
        /* base-state thermo for the energy-row scale: c_v,k, u_k and dc_v,k/dT (complex step) */
        double cv = 0.0;
        for (int k = 0; k < N; ++k) {
            double complex cpR, HRT, SR;
            nasa7_z(m, k, T[s] + I * h, &cpR, &HRT, &SR);
            cvk[k] = (creal(cpR) - 1.0) * PJO_R / m->W[k];
            uk[k] = (creal(HRT) - 1.0) * PJO_R * T[s] / m->W[k];
            dcvk[k] = cimag(cpR) / h * PJO_R / m->W[k];
            cv += Ys[k] * cvk[k];
        }
        /* one step along Y_N: its derivative enters every species column */
        for (int k = 0; k < N; ++k) Yz[k] = Ys[k];
        Yz[N - 1] += I * h;
        source_terms_cv_z(m, T[s], r0, Yz, fz, qfz, qrz, wkz);
        for (int row = 0; row < N + 1; ++row) dfN[row] = cimag(fz[row]) / h;
        for (int i = 0; i < R; ++i) {
            aqfN[i] = fabs(cimag(qfz[i]) / h);
            aqrN[i] = fabs(cimag(qrz[i]) / h);
        }
        for (int col = 0; col < N + 1; ++col) {
            if (col == N) {
                for (int row = 0; row < N + 1; ++row) {
                    Jo[(size_t)row * (N + 1) + col] = 0.0;
                    if (Jso) Jso[(size_t)row * (N + 1) + col] = 0.0;
                }
                continue;
            }
            double complex Tz = T[s];
            for (int k = 0; k < N; ++k) Yz[k] = Ys[k];
            if (col == 0) Tz += I * h;
            else Yz[col - 1] += I * h;
            source_terms_cv_z(m, Tz, r0, Yz, fz, qfz, qrz, wkz);
            for (int row = 0; row < N + 1; ++row)
                Jo[(size_t)row * (N + 1) + col] = cimag(fz[row]) / h - (col == 0 ? 0.0 : dfN[row]);
            if (!Jso) continue;
            /* scales: sum_i |nu_ki| (|d qf_i| + |d qr_i|) per species, over the column's directions */
            for (int k = 0; k < N; ++k) sk[k] = 0.0;
            for (int i = 0; i < R; ++i) {
                const pjo_rxn *r = &m->rx[i];
                double d = fabs(cimag(qfz[i]) / h) + fabs(cimag(qrz[i]) / h);
                if (col > 0) d += aqfN[i] + aqrN[i];
                for (int q = 0; q < r->nnet; ++q) sk[r->netsp[q]] += fabs(r->netnu[q]) * d;
            }
            double e0 = 0.0;
            for (int k = 0; k < N; ++k) {
                Jso[(size_t)(1 + k) * (N + 1) + col] = m->W[k] / r0 * sk[k];
                const double omk = f[1 + k] * r0 / m->W[k];
                e0 += fabs(uk[k] * m->W[k]) * sk[k] + (col == 0 ? fabs(cvk[k] * m->W[k] * omk) : 0.0);
            }
            double dcv = 0.0;
            if (col == 0)
                for (int k = 0; k < N; ++k) dcv += fabs(Ys[k] * dcvk[k]);
            else
                dcv = fabs(cvk[col - 1]) + fabs(cvk[N - 1]);
            Jso[col] = e0 / (r0 * cv) + fabs(f[0]) * dcv / cv;
        }
        free(Yz);
        free(bd);
    }
    return err ? PJO_ENOMEM : PJO_OK;
}

/* Complex-step Jacobian of the templated source terms: column 0 from T + i h, column j from
 * Y_j + i h, Y_N - i h (j = 1..N-1); column N is zero. Exact to rounding for analytic f. */
int pjo_jacobian_complex_step(const pjo_mech *m, int64_t n, const double *T, const double *P, const double *Y,
                              int64_t ldy, double h, double *jac, int64_t ldj)
{
    if (!m || n < 0 || ldy < m->ns || !(h > 0.0)) return PJO_EINVAL;
    const int N = m->ns;
    if (ldj < (int64_t)(N + 1) * (N + 1)) return PJO_EINVAL;
    if (n == 0) return PJO_OK;
    if (!T || !P || !Y || !jac) return PJO_EINVAL;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(pjo_max_threads())
    for (int64_t s = 0; s < n; ++s) {
        double complex *Yz = malloc(((size_t)N + (N + 1) + 6 * (size_t)N + 2 * (size_t)m->nr + 8) * sizeof(double complex));
        if (!Yz) { err = 1; continue; }
        double complex *fz = Yz + N, *wk = fz + N + 1;
        double *Jo = jac + s * ldj;
        const double *Ys = Y + s * ldy;
        for (int col = 0; col < N + 1; ++col) {
            double complex Tz = T[s];
            for (int k = 0; k < N; ++k) Yz[k] = Ys[k];
            if (col == 0) Tz += I * h;
            else if (col < N) { Yz[col - 1] += I * h; Yz[N - 1] -= I * h; }
            if (col < N) source_terms_z(m, Tz, P[s], Yz, fz, NULL, wk);
            for (int row = 0; row < N + 1; ++row) Jo[(size_t)row * (N + 1) + col] = (col < N) ? cimag(fz[row]) / h : 0.0;
        }
        free(Yz);
    }
    return err ? PJO_ENOMEM : PJO_OK;
}

/* ---------------------------------------------------------------------------------------------
 * Molar-concentration basis at constant pressure (conc_rhs in source_terms.inc): the source terms
 * f = (dT/dt, dV/dt, dn_1/dt..dn_{N-1}/dt) of states (T, V, n_1..n_{N-1}) at fixed P, and their
 * Jacobian by the plain definition, d f / d (T, V, n_1..n_{N-1}), one complex-step derivative per
 * column (T + i h; V (1 + i h); n_j + i h V, which moves [X_j] by i h and, through n_N, [X_N] by
 * -i h). State-major; nmol[s * ldn + k] = n_k (k < N-1). */
int pjo_eval_dydt_conc(const pjo_mech *m, int64_t n, const double *T, const double *P, const double *V,
                       const double *nmol, int64_t ldn, double *dydt, int64_t ldd)
{
    if (!m || n < 0 || ldn < m->ns - 1 || ldd < m->ns + 1) return PJO_EINVAL;
    if (n == 0) return PJO_OK;
    if (!T || !P || !V || !nmol || !dydt) return PJO_EINVAL;
    const int N = m->ns;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(pjo_max_threads())
    for (int64_t s = 0; s < n; ++s) {
        double *wk = malloc((6 * (size_t)N + (size_t)m->nr) * sizeof(double));
        if (!wk) { err = 1; continue; }
        conc_rhs_d(m, T[s], P[s], V[s], nmol + s * ldn, dydt + s * ldd, NULL, wk);
        free(wk);
    }
    return err ? PJO_ENOMEM : PJO_OK;
}

/* jac: (N+1) x (N+1) per state, rows and columns in state order (T, V, n_1..n_{N-1}); dydt
 * (optional): f. The optional scales bound the rounding of each entry for an evaluation that
 * forms it from per-reaction partial derivatives in the concentrations [X_l] (each at fixed
 * T and fixed other [X]) and in T: per reaction a_i = |c R_f| + |c R_r|, g_il = |d(c R_f)/d[X_l]| +
 * |d(c R_r)/d[X_l]|, t_i = |d(c R_f)/dT| + |d(c R_r)/dT| + (3 + orders + 6 [third body]) a_i / T;
 * per species m_kl = sum_i |nu_ki| g_il; a species entry in column n_j takes m_kj + m_kN, its V
 * entry sV_k = sum_i |nu_ki| a_i + sum_l [X_l] m_kl + [M] m_kN, its T entry
 * V (sum_i |nu_ki| t_i + sV_k / T); the T and V rows take the same sums weighted as in their
 * definitions (|H_k|, 1/(V rho c_p), 1/[M]), plus the magnitudes of their thermodynamic terms. */
int pjo_jacobian_conc(const pjo_mech *m, int64_t n, const double *T, const double *P, const double *V,
                      const double *nmol, int64_t ldn, double *jac, int64_t ldj, double *jac_scale,
                      double *dydt, int64_t ldd, double *dydt_scale)
{
    if (!m || n < 0 || ldn < m->ns - 1) return PJO_EINVAL;
    const int N = m->ns, R = m->nr;
    if (ldj < (int64_t)(N + 1) * (N + 1)) return PJO_EINVAL;
    if ((dydt || dydt_scale) && ldd < N + 1) return PJO_EINVAL;
    if (n == 0) return PJO_OK;
    if (!T || !P || !V || !nmol || !jac) return PJO_EINVAL;
    const double h = 1e-30;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(pjo_max_threads())
    for (int64_t s = 0; s < n; ++s) {
        const size_t nwk = 9 * (size_t)N + (size_t)R + 2;
        /* complex: n, f, workspace (conc_rhs and the constant-volume source terms), qf, qr, Y */
        double complex *z = malloc(((size_t)N + (N + 1) + nwk + 2 * (size_t)R + N) * sizeof(double complex));
        /* real: f, X, Y, H, cp, dcp, a, t, mN, ml, sV, sT, |omega|, column scales of the T row */
        double *b = malloc(((size_t)(N + 1) + 11 * (size_t)N + 2 * (size_t)R + (size_t)(N + 1)) * sizeof(double));
        if (!z || !b) { free(z); free(b); err = 1; continue; }
        double complex *nz = z, *fz = nz + N, *wkz = fz + N + 1, *qfz = wkz + nwk, *qrz = qfz + R, *Yz = qrz + R;
        double *f = b, *X = f + N + 1, *Y = X + N, *Hm = Y + N, *cpm = Hm + N, *dcpm = cpm + N, *ar = dcpm + N;
        double *tr = ar + R, *mN = tr + R, *ml = mN + N, *sV = ml + N, *sT = sV + N, *aom = sT + N, *sTr = aom + N;
        const double Ts = T[s], Ps = P[s], Vs = V[s], *ns_ = nmol + s * ldn;
        double *Jo = jac + s * ldj, *Jso = jac_scale ? jac_scale + s * ldj : NULL;
        const size_t ld = (size_t)N + 1;
        /* f and the columns */
        for (int k = 0; k < N - 1; ++k) nz[k] = ns_[k];
        conc_rhs_z(m, Ts, Ps, Vs, nz, fz, NULL, wkz);
        for (int r = 0; r <= N; ++r) f[r] = creal(fz[r]);
        if (dydt) for (int r = 0; r <= N; ++r) dydt[s * ldd + r] = f[r];
        for (int col = 0; col <= N; ++col) {
            double complex Tz = Ts, Vz = Vs;
            double dh = h;
            for (int k = 0; k < N - 1; ++k) nz[k] = ns_[k];
            if (col == 0) Tz += I * h;
            else if (col == 1) { Vz += I * h * Vs; dh = h * Vs; }
            else { nz[col - 2] += I * h * Vs; dh = h * Vs; }
            conc_rhs_z(m, Tz, Ps, Vz, nz, fz, NULL, wkz);
            for (int r = 0; r <= N; ++r) Jo[(size_t)r * ld + col] = cimag(fz[r]) / dh;
        }
        if (Jso || dydt_scale) {
            /* concentrations, mass fractions and molar thermodynamics of the state */
            const double M = Ps / (PJO_R * Ts);
            double sx = 0.0, rho = 0.0;
            for (int k = 0; k < N - 1; ++k) { X[k] = ns_[k] / Vs; sx += X[k]; }
            X[N - 1] = M - sx;
            for (int k = 0; k < N; ++k) rho += X[k] * m->W[k];
            for (int k = 0; k < N; ++k) Y[k] = X[k] * m->W[k] / rho;
            double K = 0.0, dK = 0.0;
            for (int k = 0; k < N; ++k) {
                double complex cpR, HRT, SR;
                nasa7_z(m, k, Ts + I * h, &cpR, &HRT, &SR);
                Hm[k] = creal(HRT) * PJO_R * Ts;
                cpm[k] = creal(cpR) * PJO_R;
                dcpm[k] = cimag(cpR) / h * PJO_R;
                K += X[k] * cpm[k];
                dK += fabs(X[k] * dcpm[k]);
            }
            /* per reaction: a_i and t_i (T-partials at fixed [X], constant-volume source terms) */
            for (int k = 0; k < N; ++k) Yz[k] = Y[k];
            source_terms_cv_z(m, Ts + I * h, rho, Yz, fz, qfz, qrz, wkz);
            for (int i = 0; i < R; ++i) {
                const pjo_rxn *r = &m->rx[i];
                int ord = 3 + (r->kind == PJO_THIRD || r->kind == PJO_FALLOFF || r->kind == PJO_CHEM ? 6 : 0);
                for (int q = 0; q < r->nr; ++q) ord += r->rnu[q];
                for (int q = 0; q < r->np; ++q) ord += r->pnu[q];
                ar[i] = fabs(creal(qfz[i])) + fabs(creal(qrz[i]));
                tr[i] = fabs(cimag(qfz[i]) / h) + fabs(cimag(qrz[i]) / h) + ord * ar[i] / Ts;
            }
            for (int k = 0; k < N; ++k) { aom[k] = 0.0; sV[k] = 0.0; sT[k] = 0.0; }
            for (int i = 0; i < R; ++i) {
                const pjo_rxn *r = &m->rx[i];
                for (int q = 0; q < r->nnet; ++q) {
                    aom[r->netsp[q]] += fabs(r->netnu[q]) * ar[i];
                    sT[r->netsp[q]] += fabs(r->netnu[q]) * tr[i];
                }
            }
            /* m_kl for l = N first (every column's second direction), then l = 1..N-1 */
            for (int l = N - 1; l >= 0; --l) {
                double *mk = (l == N - 1) ? mN : ml;
                for (int k = 0; k < N; ++k) Yz[k] = Y[k];
                Yz[l] += I * h * m->W[l] / rho;                /* [X_l] + i h */
                source_terms_cv_z(m, Ts, rho, Yz, fz, qfz, qrz, wkz);
                for (int k = 0; k < N; ++k) mk[k] = 0.0;
                for (int i = 0; i < R; ++i) {
                    const pjo_rxn *r = &m->rx[i];
                    const double g = fabs(cimag(qfz[i]) / h) + fabs(cimag(qrz[i]) / h);
                    for (int q = 0; q < r->nnet; ++q) mk[r->netsp[q]] += fabs(r->netnu[q]) * g;
                }
                for (int k = 0; k < N; ++k) sV[k] += X[l] * mk[k];
                if (l == N - 1 || !Jso) continue;
                double sh = 0.0, sn = 0.0;                     /* column n_l: species, T and V rows */
                for (int k = 0; k < N; ++k) {
                    const double skj = mk[k] + mN[k];
                    if (k < N - 1) Jso[(size_t)(2 + k) * ld + 2 + l] = skj;
                    sh += fabs(Hm[k]) * skj;
                    sn += skj;
                }
                const double sTj = (sh + fabs(f[0]) * (fabs(cpm[l]) + fabs(cpm[N - 1]))) / (Vs * K);
                sTr[2 + l] = sTj;
                Jso[2 + l] = sTj;
                Jso[ld + 2 + l] = Vs / Ts * sTj + sn / M;
            }
            double aO = 0.0, sHV = 0.0, sHT = 0.0, sVs = 0.0, sTs = 0.0, cpo = 0.0;
            for (int k = 0; k < N; ++k) {
                sV[k] += aom[k] + M * mN[k];
                sT[k] += sV[k] / Ts;                           /* per unit volume */
                aO += aom[k];
                sHV += fabs(Hm[k]) * sV[k];
                sHT += fabs(Hm[k]) * sT[k];
                sVs += sV[k];
                sTs += sT[k];
                cpo += fabs(cpm[k]) * aom[k];
            }
            if (dydt_scale) {
                double *fs = dydt_scale + s * ldd, sh = 0.0;
                for (int k = 0; k < N; ++k) sh += fabs(Hm[k]) * aom[k];
                fs[0] = sh / K;
                fs[1] = Vs * (fs[0] / Ts + aO / M);
                for (int k = 0; k < N - 1; ++k) fs[2 + k] = Vs * aom[k];
            }
            if (Jso) {
                for (int k = 0; k < N - 1; ++k) {
                    Jso[(size_t)(2 + k) * ld + 0] = Vs * sT[k];
                    Jso[(size_t)(2 + k) * ld + 1] = sV[k];
                }
                const double sTV = (sHV + fabs(f[0]) * (K + M * fabs(cpm[N - 1]))) / (Vs * K);
                const double sTT = (cpo + sHT + fabs(f[0]) * (dK + fabs(cpm[N - 1]) * M / Ts)) / K;
                Jso[0] = sTT;
                Jso[1] = sTV;
                Jso[ld + 0] = Vs * (sTT / Ts + fabs(f[0]) / (Ts * Ts) + aO / (M * Ts) + sTs / M);
                Jso[ld + 1] = fabs(f[0]) / Ts + Vs / Ts * sTV + sVs / M;
            }
        }
        free(z);
        free(b);
    }
    return err ? PJO_ENOMEM : PJO_OK;
}
