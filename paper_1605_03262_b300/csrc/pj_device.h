// Definitions shared by the host code and the device code of the B300 library: the device image
// of a kinetic model and the kernel parameter blocks. Device-only users (the runtime-compiled
// specialised kernels) include this without any host headers.
#pragma once

#ifndef __CUDACC_RTC__
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#else
typedef unsigned char uint8_t;
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef unsigned long long uintptr_t;
#endif

#include "pj_fastmath.cuh"

namespace pj {

constexpr double kR = 8.31446261815324;   // J/(mol K)
constexpr double kPatm = 101325.0;        // Pa
constexpr int kMaxSlots = 4;              // distinct species per side of a reaction
constexpr int kMaxNu = 4;                 // stoichiometric coefficient bound
constexpr int kThermoStride = 36;         // doubles per species: two ranges x 18
constexpr int kNuBias = 64;               // coefficient code = nu + kNuBias (7 bits)

enum Kind : uint8_t { kElem = 0, kThird = 1, kFalloff = 2, kChem = 3, kPlog = 4, kCheb = 5 };
enum Rev : uint8_t { kIrrev = 0, kRevKc = 1, kRevExplicit = 2 };
enum FType : uint8_t { kLindemann = 0, kTroe = 1, kSri = 2 };
enum TbMode : uint8_t { kTbNone = 0, kTbMix = 1, kTbSpecies = 2 };
enum KForm : uint8_t { kKfGeneral = 0, kKfConst = 1, kKfIntPow = 2 };

// One reaction of the device image (class-sorted order). 64 bytes.
struct alignas(16) RxnDev {
    uint8_t kind, rev, ftype, tbmode;
    uint8_t nr, np, kform, flags;        // flags bit0: Troe T** term present
    int16_t rsp[kMaxSlots];              // reactant species (distinct)
    int16_t psp[kMaxSlots];              // product species (distinct)
    int8_t rnu[kMaxSlots];
    int8_t pnu[kMaxSlots];
    int16_t tbsp;                        // third-body species m (tbmode == kTbSpecies)
    int16_t neff;                        // number of non-unity efficiencies (tbmode == kTbMix)
    int32_t eff_off;                     // offset into eff_sp / eff_eps
    int32_t par_off;                     // offset into the parameter pool
    int32_t slot_off;                    // first b-slot of this reaction
    int32_t nslot;                       // number of b-slots (species whose column this reaction touches)
    int32_t kpow;                        // integer temperature exponent (kform == kKfIntPow)
    int32_t pad;
};
static_assert(sizeof(RxnDev) == 64, "RxnDev layout");

// Pointers into one device allocation holding a model's image.
struct DevModel {
    int N, R, nslot, nnz, ncontrib, ncolent;
    const RxnDev *rx;
    const double *par;        // parameter pool
    const int *eff_sp;
    const double *eff_eps;    // alpha - 1
    const int *slot_info;     // species | (reactant slot + 1) << 16 | (product slot + 1) << 24
    const double *slot_eps;   // epsilon of the slot species in this reaction
    const double *thermo;     // N x kThermoStride
    const double *Tmid;
    const double *W;
    const double *invW;
    const double *Delta;      // 1/W_j - 1/W_N (0 for j = N-1)
    const int *sp_ptr;        // species gather CSR (N + 1)
    const int *sp_rxn;
    const double *sp_nu;
    const int *col_ptr;       // energy-row column CSR over b-slots (N + 1)
    const int *col_slot;
    const int *col_rxn;
    const int *row_ptr;       // sparse block rows (N + 1) over nnz entries
    const int *nnz_col;
    const int *nnz_cptr;      // contributions CSR (nnz + 1)
    const double *nnz_wr;     // W_k / W_j
    const int *con_slot;
    const double *con_nu;
    const int *colN_nnz;      // per row k: nnz index of column N-1, or -1
    double lnPatmR;           // ln(p_atm / R)
    // Lane-balanced schedules (see pj_model.cu). Records are lane-interleaved (chunk offset +
    // 32 t + lane is the lane's t-th item). Species gather (8 bytes) and column sums (16 bytes):
    // x = index (24 bits) | coefficient code (7 bits) << 24 | end-of-sum flag (bit 31), y = the
    // destination of the sum the item ends, z = the item's reaction (column sums). Rows and C_k
    // (16 bytes): x = index | first-item flag (bit 30) | end flag (bit 31), y = the sum's
    // destination, z, w = the item's coefficient (scale times nu) as a double.
    int rpc, n_row_chunks;    // rows per staged chunk, chunks covering the N+1 rows
    int ng, nh, ncc;          // chunks of the species-gather, column-sum and C_k schedules
    int ngp, nhp, ncp;        // pieces of the species-gather, column-sum and C_k lists (partial sums)
    const int *g_pfirst, *h_pfirst, *c_pfirst;   // per species / column: first piece (N + 1 entries)
    const uint2 *g_rec;               // species gather
    const uint4 *h_rec, *c_rec, *s_rec;   // column sums, C_k, sparse rows
    const int2 *g_chunk, *h_chunk, *c_chunk, *s_chunk;   // per chunk: record offset, rows
    int s_npart;              // partial slots a warp needs for the split row entries of one chunk
    const int2 *s_comb_chunk; // per row chunk: its first combine pass, number of passes
    // combine passes of the split row entries, one record per lane: x = the element the lane
    // loads (>= 0: staged position of the entry's value; < 0: -1 - partial slot), y = position
    // in the entry's segment | segment length << 8 | tree levels of the pass << 16
    const int2 *s_comb;
    const MathTables *tables;  // exp/log tables (pj_fastmath.cuh)
    // molar-concentration basis: per species row k < N-1, its pattern entries cc_ptr[k]..cc_ptr[k+1]
    // (columns n_j, ascending j, in cc_col; cc_wr = W_j / W_k). rx_dnu: sum_k nu_ki per reaction.
    int cc_nnz;
    const int *cc_ptr, *cc_col;
    const double *cc_wr, *rx_dnu;
    // the whole image (every array above lies in it): 256-byte aligned, image_bytes a multiple of 16
    const char *image;
    long long image_bytes;
};

// Doubles of one warp's row stage: rpc staged rows and the partial slots of split entries.
__host__ __device__ inline int row_stride(const DevModel &m) { return (m.rpc * (m.N + 1) + m.s_npart + 2) & ~1; }

// Offsets (in doubles) of one state's scratch in shared memory.
struct Scratch {
    int C, B, dB, H, cpk, Jk0, A, Ck, f, HS, red, scal, q, th, a, dH, b, rows, part, total;
    int rows_per_chunk;       // rows staged per warp chunk
};

struct KParams {
    DevModel m;
    Scratch sc;
    long long n;
    const double *T, *P, *Y;
    long long ldy;
    double *jac;
    long long ldj;
    double *dydt;
    long long ldd;
    int groups;               // states processed concurrently per CTA
    int shared_const;         // doubles of per-CTA constants at the start of shared memory
    const double *V;          // volumes (molar-concentration basis only)
};

// Batched form: one entry per (model, state batch) of a plan, and tiles of consecutive states.
struct BatchIO {
    const double *T, *P, *Y;
    long long ldy;
    double *jac;
    long long ldj;
    double *dydt;
    long long ldd;
    const double *V;          // volumes (molar-concentration basis only)
};

struct BatchItem {
    const DevModel *m;        // device copy of the model's DevModel
    Scratch sc;
    BatchIO io;
    int wps, groups, shared_const, pad;
};

struct BatchTile {
    int item, pad;
    long long begin, count;
};

struct BatchParams {
    const BatchItem *items;
    const BatchTile *tiles;
    int ntiles;
    int *counter;             // tile counter, zeroed before every launch
};

}  // namespace pj
