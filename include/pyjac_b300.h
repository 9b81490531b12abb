/*
 * pyjac_b300: batched FP64 chemical source terms and analytical constant-pressure Jacobian on
 * NVIDIA B300 (sm_103a). C ABI of libpyjacb300.so.
 *
 * The operations are those of Niemeyer, Curtis & Sung, "pyJac: analytical Jacobian generator for
 * chemical kinetics" (arXiv:1605.03262):
 *   - source terms f = dPhi/dt of the constant-pressure composition vector, Eqs. e:ode and e:dTdt
 *     (Section 2.1), with thermodynamics of Section 2.2 (Eqs. e:cpk, e:hk, e:sk) and reaction rates
 *     of Section 2.3 (Arrhenius Eq. e:arrhenius, third-body, Lindemann/Troe/SRI falloff and
 *     chemically activated reactions Eq. e:rxn_pressure, PLOG Eq. e:plog, Chebyshev Eq. e:cheb,
 *     reverse rates via the equilibrium constant Eq. e:kri or explicit Arrhenius parameters);
 *   - the analytical Jacobian J = df/dPhi of Section 3 (Eqs. e:jac_spec, e:jac_dydt, e:jac_dydy,
 *     e:jac_dt), evaluated in the reuse order of Section 4 (Algorithm 2).
 *
 * Conventions for every evaluation entry point:
 *   - Units are SI: T in K, P in Pa, mass fractions Y dimensionless, time in s.
 *   - A state is (T, P, Y_1..Y_N). All N mass fractions are read and used as given; Y_N is not
 *     recomputed from the others.
 *   - dydt: N+1 doubles per state, {dT/dt, dY_1/dt, ..., dY_N/dt}.
 *   - jac: (N+1)^2 doubles per state, row-major. Row/column 0 is temperature, rows/columns 1..N are
 *     species 1..N. Column j (1 <= j <= N-1) is the derivative along Y_j with Y_N = 1 - sum of the
 *     others (Eq. e:y_nsp), i.e. d/dY_j - d/dY_N at fixed T and P. Column N is identically zero
 *     because Y_N is not a state variable; row N is the last species (the paper's placeholder row).
 *   - Batched arrays are state-major: state s of Y starts at Y + s*ldy, of dydt at dydt + s*ldd,
 *     of jac at jac + s*ldj (leading dimensions in doubles).
 *   - Pointers of the plain entry points are device pointers on the model's device; they must be
 *     8-byte aligned. The caller owns every state and output buffer.
 *   - Evaluation is asynchronous on the given CUDA stream (cudaStream_t passed as void*; NULL = the
 *     legacy default stream). Arguments are checked on the host before any launch. There is no
 *     device-side validation of physical inputs: non-finite or non-positive inputs give non-finite
 *     outputs.
 *   - Results are deterministic: a state's outputs are bitwise identical whatever the batch it is
 *     evaluated in and whatever launch shape is configured.
 *
 * Status codes: every int-returning function returns PJ_OK or a negative PJ_E* code; the calling
 * thread's last error message is available from pj_last_error().
 */
#ifndef PYJAC_B300_H
#define PYJAC_B300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PJ_API __attribute__((visibility("default")))
#else
#define PJ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define PJ_OK 0
#define PJ_EINVAL (-1)       /* invalid argument (null pointer, bad size, stride or alignment) */
#define PJ_EFORMAT (-2)      /* malformed or truncated model buffer */
#define PJ_ECUDA (-3)        /* a CUDA runtime call failed; the message names it */
#define PJ_ENOMEM (-4)       /* host or device allocation failed */
#define PJ_ETIMEOUT (-5)     /* a bounded device wait gave up */
#define PJ_EUNSUPPORTED (-6) /* valid model outside what the kernels support (sizes, slots) */

typedef struct pj_mech pj_mech;

/* Library version (major * 10000 + minor * 100 + patch). */
PJ_API int pj_version(void);

/* Message of the last failed call on the calling thread ("" if none). The pointer stays valid
 * until the next call on the same thread. */
PJ_API const char *pj_last_error(void);

/*
 * Load a kinetic model from the binary model format (magic "PYJACMEC", version 1; species with
 * molecular weights and two-range NASA7 coefficients, reactions with stoichiometry, pressure
 * dependence, reversibility, third-body efficiencies, falloff, PLOG and Chebyshev parameters; all
 * SI). The model's device image is built on the current CUDA device; buf is only read during the
 * call. On success *out owns that device memory until pj_mech_free. Errors: PJ_EINVAL (null
 * arguments), PJ_EFORMAT (malformed buffer), PJ_EUNSUPPORTED (more than 4 distinct species on one
 * side of a reaction or a stoichiometric coefficient above 4), PJ_ECUDA / PJ_ENOMEM.
 */
PJ_API int pj_mech_load(const void *buf, size_t len, pj_mech **out);

/* pj_mech_load on the contents of a file. */
PJ_API int pj_mech_load_file(const char *path, pj_mech **out);

/* Release a model and its device memory. NULL is ignored. The caller must make sure no evaluation
 * that uses the model is still running on any stream. */
PJ_API void pj_mech_free(pj_mech *m);

/* Sizes of a loaded model: number of species N, reactions, bytes of its device image. Any output
 * pointer may be NULL. */
PJ_API int pj_mech_info(const pj_mech *m, int *n_species, int *n_reactions, size_t *dev_bytes);

/*
 * Source terms f (Eqs. e:ode, e:dTdt) for n states. T[n], P[n], Y[n][ldy >= N] in, dydt[n][ldd >= N+1]
 * out; device pointers; asynchronous on stream. n == 0 is a no-op. Errors: PJ_EINVAL (null model or
 * pointer, n < 0, ldy < N, ldd < N+1, misaligned or host pointer), PJ_ECUDA (launch failure).
 */
PJ_API int pj_eval_dydt(const pj_mech *m, int64_t n, const double *T, const double *P, const double *Y, int64_t ldy,
                 double *dydt, int64_t ldd, void *stream);

/*
 * Analytical Jacobian (Section 3, evaluated in the Section 4 reuse order) for n states, and
 * optionally the source terms. T[n], P[n], Y[n][ldy >= N] in; jac[n][ldj >= (N+1)^2] out; dydt may
 * be NULL, else dydt[n][ldd >= N+1] out. Device pointers; asynchronous on stream. Errors as
 * pj_eval_dydt, plus PJ_EINVAL for ldj < (N+1)^2 and PJ_EUNSUPPORTED when one state's working set
 * does not fit in shared memory.
 */
PJ_API int pj_eval_jacobian(const pj_mech *m, int64_t n, const double *T, const double *P, const double *Y,
                     int64_t ldy, double *jac, int64_t ldj, double *dydt, int64_t ldd, void *stream);

/*
 * Constant-volume form (Section 3.3: the density is held fixed instead of the pressure). State
 * (T, rho, Y): rho[n] in kg/m^3 replaces P[n]; p = rho R T / W follows from the ideal-gas law
 * (Eq. e:state) for the pressure-dependent rates, and [X_k] = rho Y_k / W_k. Source terms:
 * dY_k/dt = W_k omega_k / rho as at constant pressure, and dT/dt = -sum_k u_k W_k omega_k / (rho c_v)
 * with the mass-specific internal energies u_k = h_k - R T / W_k and c_v = sum_k Y_k (c_p,k - R/W_k).
 * The Jacobian is d(T, Y_1..Y_N)/dt with respect to (T, Y_1..Y_N) at fixed rho, in the same layout
 * and column convention as pj_eval_jacobian (columns j move Y_j against Y_N; column N is zero).
 * Same argument, pointer and error rules as pj_eval_dydt / pj_eval_jacobian, with the same launch
 * shapes (pj_set_launch applies to both forms).
 */
PJ_API int pj_eval_dydt_cv(const pj_mech *m, int64_t n, const double *T, const double *rho, const double *Y,
                           int64_t ldy, double *dydt, int64_t ldd, void *stream);
PJ_API int pj_eval_jacobian_cv(const pj_mech *m, int64_t n, const double *T, const double *rho, const double *Y,
                               int64_t ldy, double *jac, int64_t ldj, double *dydt, int64_t ldd, void *stream);

/*
 * Molar-concentration basis at constant pressure, as a sparse Jacobian: the formulation the paper
 * names as future work (Section 3.4, where it says the concentration basis makes the constant-
 * pressure Jacobian far sparser, and Section 6). State (T, V, n_1..n_{N-1}) at fixed P: n_k moles of
 * species k in the volume V (m^3); n_N = P V / (R T) - sum_{k<N} n_k by the ideal-gas law, so that
 * [X_k] = n_k / V and [X_N] = P / (R T) - sum_{k<N} [X_k]. Source terms, in state order:
 *   dT/dt (Eq. e:dTdt),  dV/dt = V (dT/dt / T + (R T / P) sum_k omega_k),  dn_k/dt = V omega_k,
 * with omega_k the paper's molar production rates (Section 2). The Jacobian is
 * d(dT/dt, dV/dt, dn_k/dt) / d(T, V, n_1..n_{N-1}), an (N+1) x (N+1) matrix in CSR form with a
 * pattern fixed per model (pj_conc_pattern): rows T and V dense; species row k holds columns T, V and
 * the n_j of species that share a reaction with k (as reactant, product, third-body species or
 * non-unity efficiency), or every n_j when species N takes part in one of k's reactions.
 *
 * pj_conc_pattern: *nnz = the number of stored entries; row_ptr[N+2] and col_idx[nnz] (host
 * memory, both or neither) receive the pattern, columns ascending within a row. Errors: PJ_EINVAL.
 *
 * pj_eval_jacobian_conc: T[n] (K), P[n] (Pa), V[n] (m^3), nmol[n][ldn >= N-1] (mol) in;
 * jac[n][ldj >= nnz] out, the values of each state's CSR entries in pattern order; dydt (or NULL)
 * [n][ldd >= N+1] out, the source terms in state order. Device pointers; asynchronous on stream;
 * the launch shape is the Jacobian's (pj_set_launch which = 1). Errors: PJ_EINVAL (null model or
 * pointer, n < 0, ldn < N-1, ldj < nnz, ldd < N+1, host pointer), PJ_EUNSUPPORTED (N < 2, or one
 * state's working set does not fit in shared memory), PJ_ECUDA (launch failure).
 */
PJ_API int pj_conc_pattern(const pj_mech *m, int64_t *nnz, int32_t *row_ptr, int32_t *col_idx);
PJ_API int pj_eval_jacobian_conc(const pj_mech *m, int64_t n, const double *T, const double *P, const double *V,
                                 const double *nmol, int64_t ldn, double *jac, int64_t ldj, double *dydt,
                                 int64_t ldd, void *stream);

/*
 * End-to-end variant of pj_eval_jacobian on HOST buffers (pinned host memory gives full copy
 * bandwidth; pageable memory works but is slower). The states are processed in chunks of
 * chunk_states (<= 0: the library picks); each chunk is copied to the device, evaluated and copied
 * back, with copies and kernels of consecutive chunks overlapped on two internal streams. Device
 * staging buffers are allocated on first use and kept with the model until pj_mech_free. The call
 * is synchronous: it returns after every output is in host memory. Same argument rules as
 * pj_eval_jacobian except that the pointers are host pointers.
 */
PJ_API int pj_eval_jacobian_host(const pj_mech *m, int64_t n, const double *T, const double *P, const double *Y,
                          int64_t ldy, double *jac, int64_t ldj, double *dydt, int64_t ldd, int64_t chunk_states);

/*
 * First-order forward-difference Jacobian: the finite-difference comparison of Section 5.2
 * (Performance analysis; a first-order forward difference adapted from CVODE), evaluated with the
 * library's source-term kernel. Column c of a state's Jacobian is (f(y + h_c d_c) - f(y)) / h_c:
 * d_0 moves T; d_c (c = 1..N-1) moves Y_c by +h_c and Y_N by -h_c, the directions of the
 * analytical columns; column N is zero. h_c = 2^-26 max(|y_c|, a_c), a_0 = 1 K, a_c = 1e-10 for
 * mass fractions (CVODE's relative increment sqrt(unit roundoff) |y_c| with a fixed floor in place
 * of its error-weight term). Same layout, pointer and error rules as pj_eval_jacobian (no dydt
 * output). workspace: device memory of workspace_bytes, owned by the caller, for the perturbed
 * states and their source terms; the states are processed in chunks of as many states as it holds
 * (pj_fd_workspace_bytes gives the size for n states in one pass). PJ_EINVAL if it holds less than
 * one state or is not 8-byte aligned. Asynchronous on stream; overlapping calls must not share a
 * workspace.
 */
PJ_API int pj_fd_workspace_bytes(const pj_mech *m, int64_t n, size_t *bytes);
PJ_API int pj_eval_jacobian_fd(const pj_mech *m, int64_t n, const double *T, const double *P, const double *Y,
                               int64_t ldy, double *jac, int64_t ldj, void *workspace, size_t workspace_bytes,
                               void *stream);

/*
 * Per-model specialised kernels (the paper's per-mechanism code generation, Sections 4 and 6:
 * source generated for one mechanism and compiled for it), built at run time with NVRTC. enable != 0
 * compiles the library's evaluation kernels with every size and shared-memory offset of this model
 * and its current launch shapes (pj_set_launch) as compile-time constants, loads them on the current
 * device, and makes pj_eval_dydt / pj_eval_jacobian, the constant-volume calls and
 * pj_eval_jacobian_conc use them while
 * the launch shape stays the one they were compiled for (another shape uses the data-driven kernels;
 * call again to specialise for it). The results are bitwise those of the data-driven kernels.
 * enable == 0 releases them. Takes a few seconds. Errors: PJ_EINVAL, PJ_EUNSUPPORTED (NVRTC not
 * loadable, or a working set that does not fit in shared memory), PJ_ECUDA (compilation or loading
 * failed; the message holds the compiler log). pj_mech_spec_info reports whether the Jacobian and
 * source-term calls currently run specialised kernels, and the compile time and code size; any
 * output pointer may be NULL.
 */
PJ_API int pj_mech_specialize(pj_mech *m, int enable);
PJ_API int pj_mech_spec_info(const pj_mech *m, int *active_jacobian, int *active_dydt, double *compile_seconds,
                             size_t *cubin_bytes);

/* Launch shape of the evaluation kernels for one model (which: 0 = Jacobian, 1 = source terms).
 * warps_per_state in {1, 2, 4, 8, 16}: warps that cooperate on one state; states_per_cta: states
 * a CTA evaluates concurrently (CTA size = warps_per_state * 32 * states_per_cta <= 512; at most
 * 15 when warps_per_state > 1); ctas_per_sm: resident CTAs the grid is sized for. Results do not
 * depend on the shape. pj_set_launch returns PJ_EINVAL for shapes outside these limits or whose
 * shared memory exceeds the device's per-CTA limit. */
typedef struct {
    int warps_per_state;
    int states_per_cta;
    int ctas_per_sm;
} pj_launch;

PJ_API int pj_set_launch(pj_mech *m, int which, const pj_launch *cfg);
PJ_API int pj_get_launch(const pj_mech *m, int which, pj_launch *cfg);

/* Shared memory (bytes) one CTA of the given shape needs for this model, or PJ_EINVAL. */
PJ_API int pj_launch_smem_bytes(const pj_mech *m, int which, const pj_launch *cfg, size_t *bytes);

/*
 * Batched form: one persistent launch over several (model, state batch) items of uneven size.
 * Each item names a loaded model, its n states (device T, P, Y) and its outputs; the plan splits
 * every item into tiles of consecutive states, and the CTAs of one kernel take tiles from a shared
 * counter, evaluating each with its model's warps-per-state setting (pj_set_launch). Results are
 * those of pj_eval_jacobian / pj_eval_dydt on the same states (same arithmetic, same order).
 *
 * which: 0 = Jacobian (jac required, dydt optional), 1 = source terms (dydt required).
 * shape (may be NULL): threads_per_cta (multiple of 32, <= 512; default 512), ctas_per_sm (default
 * 1) and tile_states (states per tile; 0 = four times the states a CTA evaluates concurrently).
 * pj_batch_create checks every item like the plain entry points (PJ_EINVAL / PJ_EUNSUPPORTED),
 * copies the item table and tiles to device memory it owns, and keeps the pointers: the buffers
 * must stay valid while the plan is used. pj_batch_run resets the plan's tile counter and launches
 * on the stream, asynchronously; it allocates nothing and does not synchronise, so a run can be
 * captured into a CUDA graph and replayed. Runs of one plan must not overlap on the GPU (they share
 * the counter). pj_batch_free releases the plan (no run may be in flight).
 */
typedef struct pj_batch pj_batch;

typedef struct {
    const pj_mech *mech;
    int64_t n;
    const double *T, *P, *Y;
    int64_t ldy;
    double *jac;
    int64_t ldj;
    double *dydt;
    int64_t ldd;
} pj_batch_item;

typedef struct {
    int threads_per_cta;
    int ctas_per_sm;
    int tile_states;
} pj_batch_shape;

PJ_API int pj_batch_create(const pj_batch_item *items, int n_items, int which, const pj_batch_shape *shape,
                           pj_batch **out);

/*
 * The same plan with a shape per item (item_shapes[i] for items[i]; item_shapes may be NULL, and a
 * 0 entry takes the default): warps_per_state in {1, 2, 4, 8, 16} (default: the model's
 * pj_set_launch setting, halved while a state does not fit), states_per_cta (default and upper
 * bound: as many as the CTA's threads and shared memory allow) and tile_states (default: the
 * plan's). The autotuner of the batched form chooses these; results do not depend on them.
 * Errors as pj_batch_create, plus PJ_EINVAL for a width outside the set or wider than the CTA.
 */
typedef struct {
    int warps_per_state;
    int states_per_cta;
    int tile_states;
} pj_batch_item_shape;

PJ_API int pj_batch_create_ex(const pj_batch_item *items, int n_items, int which, const pj_batch_shape *shape,
                              const pj_batch_item_shape *item_shapes, pj_batch **out);
PJ_API int pj_batch_run(pj_batch *b, void *stream);
PJ_API int pj_batch_info(const pj_batch *b, int *n_tiles, size_t *smem_bytes, int *threads_per_cta);
PJ_API void pj_batch_free(pj_batch *b);

/*
 * The plan's kernel specialised for its models (the per-mechanism code generation of Sections 4
 * and 6, as pj_mech_specialize, for a mixed batch): enable != 0 compiles with NVRTC one persistent
 * kernel in which every distinct (model, warps per state, states per round) triple of the plan is
 * a part with that model's sizes, shared-memory offsets, group width and states per round as
 * compile-time constants and its device pointers in constant memory; the parts run one after
 * another (models in decreasing work per state; a CTA moves to the next part when the current one
 * has no tile left), and pj_batch_run launches it; enable == 0 returns to the data-driven kernel.
 * An item whose group width the plan chose (not the caller) and had to halve for shared memory
 * runs at its model's own width where that fits, and tiles of costly models are cut into shorter
 * ones. Same results, bit for bit. Takes seconds (one compile per plan); call it before capturing
 * pj_batch_run into a graph. pj_batch_spec_info reports whether the plan runs it, its number of
 * parts, the compile time and code size (any output may be NULL). Errors as pj_mech_specialize,
 * and PJ_EUNSUPPORTED for a plan of more than 64 such parts.
 */
PJ_API int pj_batch_specialize(pj_batch *b, int enable);
PJ_API int pj_batch_spec_info(const pj_batch *b, int *active, int *slots, double *compile_seconds,
                              size_t *cubin_bytes);

/*
 * Batched launch that allocates nothing (the paper has no counterpart; it serves callers, not the
 * method). Some callers cannot allocate device memory where they call us: a reacting-flow solver
 * that owns a fixed device memory pool and forbids cudaMalloc/cudaFree inside its time step
 * (those calls can synchronise the device and fragment the pool), or code that must not meet an
 * allocation failure in the middle of a run. pj_batch_run_noalloc evaluates the same items as
 * pj_batch_create + pj_batch_run would (same arithmetic, bitwise the same results), without
 * device memory of its own: the item table and the tile bounds travel to the kernel by value, in
 * its parameter block, and the one piece of device scratch -- the tile counter from which the
 * CTAs take tiles -- lies in a fixed static device array of the library (256 bytes, held by every
 * GPU that loads the library until the process exits). It calls no cudaMalloc, cudaFree or other
 * allocating routine; the caller still provides every input and output buffer.
 *
 * Limits and rules:
 *   - at most 64 items per call (the size of the parameter block); more are rejected with
 *     PJ_EINVAL and a message naming the limit; items with n = 0 are allowed anywhere in the list;
 *   - which: 0 = Jacobian (jac required, dydt optional), 1 = source terms (dydt required);
 *     tile_states: states per tile, 0 = four times the states a CTA evaluates concurrently;
 *   - every call uses the same counter, which keeps the last call's value; each call zeroes it
 *     with an asynchronous memset on the given stream before its kernel starts. Calls that
 *     overlap on the GPU race on it: order them on one stream, or wait for one to finish before
 *     issuing the next;
 *   - the first call on a device looks up the array's device address (cudaGetSymbolAddress); make
 *     that first call before any stream capture;
 *   - asynchronous on the stream: the call does not wait for earlier work on the stream, and
 *     reads nothing of the host's item array after it returns; argument errors as
 *     pj_batch_create.
 */
PJ_API int pj_batch_run_noalloc(const pj_batch_item *items, int n_items, int which, int tile_states, void *stream);

/*
 * The same launch with the tile counter in a device workspace of the caller (at least
 * pj_batch_workspace_bytes() bytes, 16-byte aligned, on the current device) instead of the
 * library's static array: calls on different workspaces may overlap on the GPU (one workspace per
 * stream, e.g. a server's pool). At most 64 items; same argument rules and errors as
 * pj_batch_run_noalloc, plus PJ_EINVAL for a missing, small, misaligned or non-device workspace.
 * Calls that share a workspace must be ordered on one stream.
 */
PJ_API size_t pj_batch_workspace_bytes(void);
PJ_API int pj_batch_run_ws(const pj_batch_item *items, int n_items, int which, int tile_states, void *workspace,
                           size_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PYJAC_B300_H */
