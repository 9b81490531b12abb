// Internal host-side definitions of the B300 library (the device-visible ones are in
// pj_device.h). Not part of the public C ABI (include/pyjac_b300.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "pj_device.h"

namespace pj {

struct LaunchCfg {
    int wps = 1;              // warps per state
    int groups = 4;           // states per CTA
    int ctas_per_sm = 1;
};

struct FormatError : std::runtime_error {
    using std::runtime_error::runtime_error;
};
struct Unsupported : std::runtime_error {
    using std::runtime_error::runtime_error;
};

// Host copy of a model's device image (pj_model.cu).
struct HostImage {
    std::vector<RxnDev> rx;
    std::vector<double> par, eff_eps, slot_eps, thermo, Tmid, W, invW, Delta, sp_nu, nnz_wr, con_nu;
    std::vector<int> eff_sp, slot_info, sp_ptr, sp_rxn, col_ptr, col_slot, col_rxn, row_ptr, nnz_col, nnz_cptr,
        con_slot, colN_nnz;
    std::vector<int> perm;
    int N = 0, R = 0, NE = 0;
    // lane-balanced schedules
    int rpc = 1, n_row_chunks = 0, ng = 0, nh = 0, ncc = 0, ngp = 0, nhp = 0, ncp = 0;
    std::vector<int> g_pfirst, h_pfirst, c_pfirst;
    std::vector<uint32_t> g_rec, h_rec, c_rec, s_rec;       // 2, 4, 4, 4 words per record
    std::vector<int> g_chunk, h_chunk, c_chunk, s_chunk;   // (record offset, rows) per chunk
    int s_npart = 0;
    std::vector<int> s_comb_chunk, s_comb;                 // (first pass, passes) per chunk; 32 x 2 ints per pass
    // molar-concentration basis: species-row pattern (DevModel::cc_ptr / cc_col / cc_wr), sum_k nu_ki
    std::vector<int> cc_ptr, cc_col;
    std::vector<double> cc_wr, rx_dnu;
};


HostImage build_image(const void *buf, size_t len);                 // throws FormatError / Unsupported
Scratch make_scratch(const DevModel &m, bool jac, int wps);
// Warps per state of the default launch shape; also the number of warps the gather schedules are
// split for (measured on B300: two warps per state up to ~100 species, then wider groups).
inline int default_wps(int N, bool jac) {
    return jac ? (N <= 24 ? 1 : N <= 96 ? 2 : N <= 200 ? 4 : 16) : (N <= 128 ? 1 : 2);
}
int shared_const_doubles(int N);
// cv: the constant-volume form, with p.P holding the densities rho instead of pressures.
cudaError_t launch_eval(const KParams &p, bool jac, bool cv, int wps, int blocks, size_t smem, cudaStream_t stream);
cudaError_t launch_conc(const KParams &p, int wps, int blocks, size_t smem, cudaStream_t stream);
cudaError_t prepare_batch_kernel(bool jac, size_t dyn_smem, size_t *static_smem);
cudaError_t launch_batch(const BatchParams &p, bool jac, int blocks, int threads, size_t smem, cudaStream_t stream);
// Forward-difference Jacobian kernels (pj_fd.cu).
cudaError_t launch_fd_perturb(int N, long long ns, const double *T, const double *P, const double *Y, long long ldy,
                              double *Tp, double *Pp, double *Yp, cudaStream_t st);
cudaError_t launch_fd_difference(int N, long long ns, const double *T, const double *Y, long long ldy,
                                 const double *F0, const double *Fp, double *jac, long long ldj, cudaStream_t st);
int set_error(int code, const std::string &msg);   // records the calling thread's last error, returns code

}  // namespace pj

struct pj_host_staging;

// Runtime-compiled kernels specialised for one model and its launch shapes (pj_nvrtc.cu).
struct pj_spec {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern[5] = {};       // source terms / Jacobian (index 2 * jac) x constant p / v (+ cv);
                                     // 4: the molar-concentration basis Jacobian
    pj::LaunchCfg jac_cfg, dydt_cfg; // the shapes they were compiled for
    double compile_seconds = 0.0;
    size_t cubin_bytes = 0;
};

struct pj_mech {
    int N = 0, R = 0, NE = 0;
    pj::DevModel dev{};
    void *dev_blob = nullptr;
    size_t dev_bytes = 0;
    std::vector<int> perm;          // sorted position -> original reaction index
    pj::LaunchCfg jac_cfg, dydt_cfg;
    int jac_cfg_set = 0, dydt_cfg_set = 0;
    int device = 0;
    pj_host_staging *staging = nullptr;   // device buffers of pj_eval_jacobian_host (lazy)
    const pj::DevModel *dev_model = nullptr;   // device copy of dev (for batched plans)
    pj_spec *spec = nullptr;        // specialised kernels (pj_mech_specialize), or none
    std::vector<int> cc_ptr, cc_col;   // molar-concentration basis: species-row pattern (host copy)
};

// Kernel of a batched plan specialised for its models (pj_nvrtc.cu): each distinct (model, warps
// per state) pair of the plan is a slot whose sizes, offsets and group width are compile-time
// constants; the kernel dispatches on the slot of a tile's item (BatchItem::pad).
struct pj_batch_spec {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    double compile_seconds = 0.0;
    size_t cubin_bytes = 0;
    int slots = 0;
    void *dev = nullptr;              // device: items | tiles of the specialised kernel
    pj::BatchItem *items = nullptr;   // the plan's items at the specialised kernel's group widths
    pj::BatchTile *tiles = nullptr;   // the plan's tiles grouped by slot, in the kernel's slot order
    size_t smem = 0;                  // its dynamic shared memory per CTA
};

// A batched plan (pj_batch.cu): launch shape, device copies of the item table and tiles, and the
// host copies the specialisation needs.
struct pj_batch {
    int which = 0;                 // 0 Jacobian, 1 source terms
    int device = 0;
    int threads = 0, ctas_per_sm = 1, sms = 0;
    size_t smem = 0;
    int ntiles = 0;
    void *dev = nullptr;           // items | tiles | counter
    pj::BatchParams params{};
    std::vector<pj::BatchItem> items;        // host copy; pad = the item's slot
    std::vector<pj::BatchTile> tiles;        // host copy, in the data-driven kernel's order
    std::vector<char> auto_width;            // per item: the plan chose its group width (the caller did not)
    std::vector<const pj_mech *> slot_mech;  // per slot: its model
    std::vector<int> slot_wps;               // per slot: warps per state
    pj_batch_spec *spec = nullptr;
};

namespace pj {
// Tile counters in a plan's device buffer: one, or one per slot for the specialised kernel, which
// is compiled for at most this many (model, group width) slots.
constexpr int kBatchSpecMaxSlots = 64;
// Static shared memory the specialised batched kernel may use (its tile and reaction-stage
// counters, one of each whatever the number of slots); the item shapes of its plan leave this much
// of the CTA's shared memory free.
constexpr size_t kSpecBatchStaticSmem = 64;
// Work of one batched tile at most, in the plans' per-state cost units (R * 60 + (N+1)^2): four
// rounds of seven states of the 53-species model, about 0.4 ms (default tiles and the specialised
// kernel's tiles; a tile length the caller sets is kept).
constexpr double kTileWork = 6.3e5;

// Group width, states per CTA and scratch of one model in a batched launch of `threads` threads
// and `budget` bytes of dynamic shared memory per CTA: the model's configured width, halved while
// it exceeds the CTA or while one state's working set does not fit. False if no width fits.
bool batch_group_shape(const pj_mech &m, bool jac, int threads, size_t budget, int *wps, int *groups, Scratch *sc);
}  // namespace pj

void pj_host_staging_release(pj_mech *m);

namespace pj {
// Specialised kernels (pj_nvrtc.cu): compile and load them for the model's current launch shapes;
// release them; the kernel for (jac, cv) if one was compiled for launch shape c, else null.
int specialize(pj_mech *m, std::string *err);
void spec_release(pj_mech *m);
int specialize_batch(pj_batch *b, std::string *err);
void batch_spec_release(pj_batch *b);
const void *spec_kernel(const pj_mech *m, bool jac, bool cv, const LaunchCfg &c);
const void *spec_conc_kernel(const pj_mech *m, const LaunchCfg &c);
constexpr int kSpecKernels = 5;
}  // namespace pj
