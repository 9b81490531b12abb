/*
 * Oracle (test infrastructure only): plain FP64 CPU evaluation of the chemical source terms and
 * their analytical constant-pressure Jacobian, written from the paper's Sections 2 and 3.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg use it; the product path
 * never does. It shares no code with the CUDA library.
 *
 * This header holds the oracle's own in-memory model, filled by its own reader of the binary
 * model format (the format is documented in the synthetic-input generator).
 */
#ifndef PJO_ORACLE_MODEL_H
#define PJO_ORACLE_MODEL_H

#include <stdint.h>
#include <stddef.h>

#define PJO_R    8.31446261815324   /* universal gas constant, J/(mol K) */
#define PJO_PATM 101325.0           /* one standard atmosphere, Pa */

enum { PJO_ELEM = 0, PJO_THIRD = 1, PJO_FALLOFF = 2, PJO_CHEM = 3, PJO_PLOG = 4, PJO_CHEB = 5 };
enum { PJO_IRREV = 0, PJO_REV_KC = 1, PJO_REV_EXPLICIT = 2 };
enum { PJO_LINDEMANN = 0, PJO_TROE = 1, PJO_SRI = 2 };
enum { PJO_TB_MIX = 1, PJO_TB_SPECIES = 2 };

#define PJO_MAXSLOT 8

typedef struct {
    int kind, rev;
    int nr, np;
    int rsp[PJO_MAXSLOT], rnu[PJO_MAXSLOT];   /* reactants: species, nu' */
    int psp[PJO_MAXSLOT], pnu[PJO_MAXSLOT];   /* products: species, nu'' */
    double A, beta, Ta;                        /* forward Arrhenius (kinds 0, 1) */
    double Ar, betar, Tar;                     /* explicit reverse Arrhenius */
    int tb_mode, tb_sp;
    double *alpha;                             /* dense third-body efficiency vector (length N) or NULL */
    double k0[3], kinf[3];                     /* falloff limits: A, beta, Ta */
    int ftype, has_T2;
    double fp[5];                              /* Troe a, T***, T*, T**; SRI a, b, c, d, e */
    int nplog;
    double *plog;                              /* nplog x (p, A, beta, Ta) */
    int nt, npc;
    double cheb_rng[4];                        /* Tmin, Tmax, Pmin, Pmax */
    double *eta;                               /* nt x npc, row-major */
    int nnet;                                  /* species with nonzero net coefficient nu = nu'' - nu' */
    int netsp[2 * PJO_MAXSLOT];
    int netnu[2 * PJO_MAXSLOT];
} pjo_rxn;

typedef struct pjo_mech {
    int ne, ns, nr;
    double *W;
    double *Tmid;
    double *alo, *ahi;     /* 7 coefficients per species */
    int *elem;             /* ns x ne */
    pjo_rxn *rx;
} pjo_mech;

#endif
