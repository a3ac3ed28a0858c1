/*
 * dso.h -- C ABI of the GB300 diabatic split-operator library.
 *
 * Propagates an S-component nuclear wavepacket psi_s(q) on a periodic
 * D-dimensional Fourier grid under the separable diabatic Hamiltonian
 * H = p^T m^{-1} p / 2 * 1 + V(q)  (Eq. (diab_mol_ham), Sec. II H of
 * Roulet, Choi, Vanicek, arXiv:1903.04946), with the second-order VTV
 * split-operator step (Eq. (so_VTV)) and its recursive symmetric triple-jump
 * and Suzuki-fractal compositions (Sec. II D-E) of orders 2..10, using the
 * pruned splitting coefficients and unique-coefficient index arrays of
 * Sec. II F (Eq. (merging_splitting_coeff_b_zero), Eq. (range_index_unq)).
 * The kinetic and potential actions are applied in the momentum and position
 * representations, switched by the library's own FFT kernels (Sec. II G).
 *
 * Conventions (all entry points):
 *  - atomic units, hbar = 1;
 *  - grid axis d has n[d] points q_k = qmin[d] + k (qmax[d]-qmin[d])/n[d],
 *    k = 0..n[d]-1 (periodic, right endpoint excluded);
 *  - psi is complex128 (interleaved re, im) in a DSO_FP64 context and
 *    complex64 in a DSO_FP32 context, surface-major [S][n_0][n_1]...[n_{D-1}],
 *    last axis contiguous;
 *  - the potential is real symmetric, passed packed as the upper triangle
 *    [S(S+1)/2][n_0]...[n_{D-1}] float64, pairs (r,c), r <= c, row-major:
 *    (0,0),(0,1),(1,1) for S = 2; (0,0),(0,1),(0,2),(1,1),(1,2),(2,2) for S = 3;
 *  - `where` arguments say where a caller buffer lives: DSO_HOST (pageable or
 *    pinned host memory) or DSO_DEVICE (device memory of the context's GPU).
 *
 * Ownership: the caller owns every buffer it passes; the library copies in
 * and out and keeps no caller pointer after a call returns.  The library
 * owns the context, its device wavefunction, operator tables and work
 * buffers, all released by dso_destroy.
 *
 * Errors: every call returns a dso_status and never aborts.  On failure the
 * context is unchanged (except for the error text) unless stated otherwise;
 * dso_last_error gives a message for the calling thread.
 *
 * Threads and streams: a context is used by one thread at a time.  All GPU
 * work of a context is issued on its stream; calls that return results to
 * host memory synchronise that stream.
 */
#ifndef DSO_H
#define DSO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dso_ctx dso_ctx;

typedef enum {
  DSO_OK = 0,
  DSO_EINVAL = -1,   /* bad argument or unsupported configuration */
  DSO_ENOMEM = -2,   /* device allocation failed */
  DSO_ECUDA = -3,    /* CUDA runtime error */
  DSO_ESTATE = -4,   /* call out of order (e.g. propagate before set_psi) */
  DSO_ETIMEOUT = -5, /* a bounded device wait gave up */
  DSO_ENUMERIC = -6  /* non-finite input or result */
} dso_status;

enum { DSO_HOST = 0, DSO_DEVICE = 1 };
enum { DSO_FP64 = 0, DSO_FP32 = 1 };
enum { DSO_TRIPLE_JUMP = 0, DSO_SUZUKI = 1, DSO_OPTIMAL = 2 };
enum { DSO_VTV = 0, DSO_TVT = 1, DSO_VT = 2, DSO_TV = 3 };
enum { DSO_KINETIC_AUTO = -1, DSO_KINETIC_JOINT = 0, DSO_KINETIC_AXES = 1 };
/* Plane pass (dso_set_plane_pass). */
enum { DSO_PLANE_AUTO = -1, DSO_PLANE_OFF = 0, DSO_PLANE_ON = 1 };
/* Potential operators (dso_set_operator_mode). */
enum { DSO_OPERATORS_AUTO = -1, DSO_OPERATORS_TABLES = 0, DSO_OPERATORS_ON_THE_FLY = 1 };

/* Limits of this build. */
#define DSO_MAX_DIM 3
#define DSO_MAX_SURFACES 4
#define DSO_MIN_AXIS 8
#define DSO_MAX_AXIS (1 << 22)      /* points on one axis, any D */
#define DSO_MAX_AXIS_1D DSO_MAX_AXIS
#define DSO_MAX_POINTS (1LL << 30)  /* grid points per surface */

/* Create a context on CUDA device `device`.  precision DSO_FP64 keeps psi,
 * the operator tables and the FFTs in FP64; DSO_FP32 stores psi and the
 * tables as complex64 and runs the FFTs in FP32, while the potential phase
 * angles V a~ dt, the kinetic phases, the composition coefficients and the
 * norm/energy reductions stay FP64 (tables are rounded to FP32 once).
 * `cuda_stream` is a cudaStream_t owned by the caller, or NULL to let the
 * context create and own a non-blocking stream.  *out receives the context
 * (NULL on failure). */
dso_status dso_create(dso_ctx** out, int device, int precision, void* cuda_stream);

/* Release the context and every device buffer it owns.  NULL is a no-op. */
void dso_destroy(dso_ctx* ctx);

/* Grid of Sec. II G / App. B: D in 1..DSO_MAX_DIM axes, n[d] a power of two
 * in [DSO_MIN_AXIS, DSO_MAX_AXIS], at most DSO_MAX_POINTS points in all,
 * qmax[d] > qmin[d] (host arrays of length D).  Resets any loaded potential,
 * masses, state and tables.  An axis longer than 4096 points (or an axis 0
 * whose S surfaces exceed 8192 points in all) is transformed as two axes of
 * n1 x n2 points with twiddles between them (a four-step FFT), which the
 * library arranges by itself; the kernel passes then run over these
 * "virtual" axes (dso_profile_steps and dso_tuned_plan number them). */
dso_status dso_set_grid(dso_ctx* ctx, int D, const int64_t* n, const double* qmin,
                        const double* qmax);

/* Batch of B independent jobs (1..2^20) on the same grid, with the same
 * masses and composition scheme but their own potentials and wavefunctions:
 * the potential becomes [B][S(S+1)/2][grid] and psi [B][S][grid], and every
 * pass of dso_propagate advances all B jobs (one launch per pass for the
 * whole batch).  Call after dso_set_grid (which resets the batch to 1) and
 * before dso_load_potential; resets potential, state and tables. */
dso_status dso_set_batch(dso_ctx* ctx, int B);

/* Diagonal mass matrix m of Eq. (diab_mol_ham): D positive values (host). */
dso_status dso_set_masses(dso_ctx* ctx, const double* m);

/* Diabatic potential V(q) of Eq. (diab_mol_ham): S in 2..DSO_MAX_SURFACES
 * surfaces, packed upper triangle as described above, finite values.
 * Copied to the device; resets the state and the tables. */
dso_status dso_load_potential(dso_ctx* ctx, int S, const double* V, int where);

/* Composition of Sec. II D-F: order in {2,4,6,8,10}; scheme DSO_TRIPLE_JUMP
 * or DSO_SUZUKI (recursive), or DSO_OPTIMAL for orders 6 and 8: the
 * non-recursive 9- and 17-stage symmetric compositions of Kahan and Li that
 * Table II lists as "optimal" (coefficients from the literature the paper
 * cites, tabulated in the library); elementary DSO_VTV (Eq. (so_VTV): the potential acts first
 * and last, with the a~ coefficients) or DSO_TVT (Eq. (so_TVT): the kinetic
 * step acts first and last and takes the a~ coefficients, the potential the
 * b~); prune must be 1 (the coefficients of Eq.
 * (merging_splitting_coeff_b_zero)).
 * The first-order algorithms of Sec. II E take order 1 (scheme ignored):
 * elementary DSO_VT (Eq. (so_VT): the kinetic step acts first, then the
 * potential) or DSO_TV (Eq. (so_TV): the potential first).  They are not
 * symmetric and are not composed; they serve as the paper's first-order
 * reference (and negative control for the geometric properties).  They run
 * on the VTV (TV) or TVT (VT) pass machinery with coefficients a = (1, 0),
 * b = (1): the trailing zero-time action is the identity up to rounding. */
dso_status dso_set_scheme(dso_ctx* ctx, int order, int scheme, int elementary, int prune);

/* Any symmetric composition of the second-order step (Sec. II D): the
 * m elementary coefficients gamma (host, time order) make one time step
 * U(dt) = U_2(gamma_m dt) ... U_2(gamma_1 dt), with U_2 the elementary
 * method DSO_VTV or DSO_TVT.  They are expanded, pruned and indexed as for
 * the built-in schemes (Secs. II E-F).  This is how the paper's "optimal"
 * compositions (Sec. II D, Table II), whose coefficients come from the
 * literature and not from a recursion, are used.  Requirements: 1 <= m <=
 * 4096, every gamma finite and nonzero, sum 1 within 1e-13, and
 * gamma_k = gamma_{m+1-k} within 1e-14 of the largest; else DSO_EINVAL.
 * The order of the result is whatever the coefficients achieve: the
 * library does not check order conditions. */
dso_status dso_set_composition(dso_ctx* ctx, int m, const double* gamma, int elementary);

/* Host-only: the pruned coefficients that dso_set_composition would use,
 * in the layout of dso_scheme_coefficients. */
dso_status dso_composition_coefficients(int m, const double* gamma, int* n_a, int* n_b, double* a, double* b,
                                        int* ia, int* ib, int* n_a_unq, int* n_b_unq);

/* Norm monitor (failure detection).  Every split-operator step is unitary,
 * so each job's norm may change only by round-off.  With tol > 0, every
 * dso_propagate compares each job's norm after the call with the norm at
 * the last dso_set_psi (or at the first checked call) and returns
 * DSO_ENUMERIC, naming the job, when they differ by more than tol relative.
 * This catches a corrupted state (non-finite values, a faulty input, a
 * hardware or software error) at the call where it appears.  A checked
 * dso_propagate synchronises its stream (one reduction of psi and a copy of
 * B numbers).  tol = 0 (the default) switches the check off; tol < 0 or
 * non-finite is DSO_EINVAL.  The paper has no counterpart. */
dso_status dso_set_norm_check(dso_ctx* ctx, double tol);

/* Diagnostics of the bounded device waits (failure detection).  The TMA
 * kernel variants wait for their tile copies on mbarriers with a bounded
 * number of polls; a wait that gives up lets every copy already started land,
 * records a code, and the next synchronising call (dso_get_psi to host
 * memory) returns DSO_ETIMEOUT.  With polls > 0, every tile of the TMA
 * variant (variant 2 of dso_tuned_plan) additionally waits, with a limit of
 * `polls`, on a barrier that no copy ever completes, so that the failure path
 * can be exercised without a fault: the wait gives up, the timeout is
 * reported, and the propagation itself is unaffected.  0 (the default)
 * switches it off.  The paper has no counterpart. */
dso_status dso_set_wait_probe(dso_ctx* ctx, int polls);

/* Device address of the context's psi ([B][S][grid], the context's element
 * type), borrowed: valid until a call that reallocates the state
 * (dso_set_grid, dso_set_batch, dso_load_potential, dso_destroy).  Lets
 * other device code read or write the state in place without a copy (for
 * example dso_position_observables_noalloc).  Writes through it bypass the
 * finite check of dso_set_psi and do not reset the norm monitor's reference,
 * so dso_set_norm_check sees them as drift.  Work on another stream must be
 * ordered with the context's stream by the caller. */
dso_status dso_psi_device_pointer(dso_ctx* ctx, void** out);

/* Set psi ([B][S][grid], complex128 or complex64 by the context's
 * precision) from host or device memory.  Host data is staged on the
 * device and checked there: a non-finite value returns DSO_ENUMERIC and
 * leaves psi unchanged; the call returns when the host buffer may be reused.
 * Device data is copied on the context's stream without a check. */
dso_status dso_set_psi(dso_ctx* ctx, const void* psi, int where);

/* Advance psi by time t with step dt (dt may be negative; t/dt must be a
 * non-negative integer within 1e-9 relative, else DSO_EINVAL).  Each step
 * applies U_V(a~_1 dt) U_T(b~_1 dt) ... U_T(b~_{N_B} dt) U_V(a~_{N_B+1} dt)
 * in the order of the general split-operator product of Sec. II E.
 * Asynchronous on the context's stream.  For DSO_TVT the roles of U_V and
 * U_T are exchanged. */
dso_status dso_propagate(dso_ctx* ctx, double t, double dt);

/* Copy psi ([S][grid], complex128 or complex64 by the context's precision)
 * to host or device memory.  A host copy synchronises the stream. */
dso_status dso_get_psi(dso_ctx* ctx, void* out, int where);

/* Observables of Sec. II A on the current psi, in FP64: norm = ||psi||,
 * energy = <psi|H|psi> (kinetic part in the momentum representation,
 * potential part in the position representation), pops[s] = ||psi_s||^2.
 * Host arrays with one entry per job (norm, energy: B entries; pops: B*S,
 * job-major).  Any output pointer may be NULL.  Synchronises the stream. */
dso_status dso_observables(dso_ctx* ctx, double* norm, double* energy, double* pops);

/* Inner product of Sec. II A, <psi|phi> = dV sum_s sum_q conj(psi_s(q))
 * phi_s(q), of the context's psi (the bra) with phi (the ket), per job: re[b]
 * and im[b] (host arrays of B entries; either may be NULL).  The symplectic
 * two-form is omega(psi, phi) = -2 im[b] (hbar = 1), and <psi|psi> is the
 * squared norm.  phi has psi's layout and element type ([B][S][grid],
 * complex128 or complex64 by the context's precision), in host memory
 * (staged in the context's work buffer) or device memory (where).  The
 * reduction is FP64 with fixed per-block partial sums added on the host in a
 * fixed order, so the result does not depend on scheduling.  A propagation is
 * unitary (Sec. II A, App. A): <U psi|U phi> = <psi|phi> to round-off.
 * Synchronises the stream. */
dso_status dso_inner(dso_ctx* ctx, const void* phi, int where, double* re, double* im);

/* The phase of each surface's wavefunction at its density maximum (the
 * wavepacket-phase observable of the convergence study, Sec. III A): for
 * every job b and surface s, index[b*S+s] receives the first flat grid index
 * (storage order) where |psi_s|^2 is largest and phase[b*S+s] = arg psi_s
 * there, in (-pi, pi].  Host arrays of B*S entries; either may be NULL.
 * Synchronises the stream. */
dso_status dso_phase_at_density_maximum(dso_ctx* ctx, int64_t* index, double* phase);

/* Pruned splitting coefficients of a composed scheme (Sec. II D-F), host
 * only (no context, no GPU): a~ has n_a = N_B + 1 entries and b~ n_b = N_B
 * (the substeps per time step); ia/ib are 0-based indices into the lists of
 * unique values (Eq. (range_index_unq)), whose lengths go to n_a_unq and
 * n_b_unq (Table II).  Output arrays may be NULL to query sizes; non-NULL
 * arrays must hold n_a (a, ia), n_b (b, ib) entries. */
dso_status dso_scheme_coefficients(int order, int scheme, int* n_a, int* n_b, double* a, double* b,
                                   int* ia, int* ib, int* n_a_unq, int* n_b_unq);

/* Diagnostics: advance psi by `nsteps` time steps of the current scheme
 * (the pass list of the steps after the first) with plain launches and a
 * CUDA event pair around every kernel on the context's stream, then report
 * per kind of pass: (virtual) axis, flags (bit 0 inverse FFT first, bit 1 forward FFT,
 * bit 2 kinetic phase + inverse FFT, bit 8 one potential unitary, bit 9 a
 * second one, bit 10 a second kinetic phase), surfaces staged per tile, launches per time step and the
 * average duration of one launch in milliseconds, and the tile line count
 * and kernel variant (0 one CTA per tile, 1 persistent with a tile queue)
 * the autotuner chose.  At most max_kinds kinds are written; *n_kinds
 * receives the number of kinds.  Any output array may be NULL.
 * Synchronises. */
dso_status dso_profile_steps(dso_ctx* ctx, double dt, int nsteps, int max_kinds, int* n_kinds, int* axis,
                             int* flags, int* surfaces, int* launches_per_step, double* avg_ms,
                             int* tile_lines, int* variant);

/* Non-blocking progress query: 1 while GPU work issued by this context is
 * still pending on its stream, 0 when all of it has finished, a negative
 * dso_status on error.  Lets a host loop serve many contexts without
 * blocking on any one of them. */
int dso_busy(const dso_ctx* ctx);

/* The kernel configuration the autotuner chose for this context, written to
 * `out` (capacity `cap` bytes, NUL-terminated) as entries
 * "axis,staged,variant,tile_lines,ctas_per_sm;" (axis: the virtual axis of
 * the passes, see dso_set_grid) where staged is 0 for passes
 * staging one surface and 1 for passes staging all S, and variant is 0 (one
 * CTA per tile), 1 (persistent, cp.async), 2 (TMA) or 3 (persistent, TMA).
 * Setting the environment variable DSO_PLAN to such a string before the
 * first propagation makes a context use that configuration instead of timing
 * the candidates (entries that do not fit the grid are ignored), so that a
 * profiler run can reproduce the configuration of a timed run.  Returns the
 * length written, or a negative dso_status (DSO_EINVAL if cap is too small). */
int dso_tuned_plan(const dso_ctx* ctx, char* out, int cap);

/* Number of kernel launches this context has issued since creation
 * (diagnostics: counts each launch of the library's own kernels, including
 * those inside CUDA-graph replays). */
int64_t dso_launch_count(const dso_ctx* ctx);

/* Allocation-free populations and potential energy of a device
 * wavefunction.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory themselves or let a library do
 * it (code running under a pool allocator that owns all device memory, an
 * engine whose memory budget is fixed before it starts, a context where an
 * allocation would synchronise the device).  It calls no cudaMalloc or
 * cudaFree and needs no context: its per-block partial sums live in a
 * file-scope device array of 304 x 8 doubles (19,456 bytes) that every GPU
 * loading this library holds until the process exits.
 *
 * psi: device pointer, complex128 [S][P] (position representation);
 * V: device pointer to the packed potential [S(S+1)/2][P], or NULL to skip
 * the potential term; S in 1..4 (larger S does not fit the scratch array
 * and returns DSO_EINVAL); P >= 1 grid points per surface; dV the grid cell
 * volume; out: device pointer to S + 1 doubles receiving
 * out[s] = dV sum_q |psi_s(q)|^2 and out[S] = dV sum_q Re psi^dagger V psi
 * (0 when V is NULL).  Runs on `cuda_stream` (a cudaStream_t, NULL for the
 * legacy default stream) on the calling thread's current device and does
 * not synchronise.
 *
 * psi must be 16-byte aligned and V and out 8-byte aligned (DSO_EINVAL
 * otherwise: a misaligned element pointer would fault the kernel).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress with that device current); make that first call
 * before capturing the stream into a CUDA graph.  The address is kept with
 * the device's driver context and looked up again when that context changes
 * (for example after cudaDeviceReset); a call that is captured into a graph
 * keeps the address of the context it was captured in.  Every call on a device
 * shares the one array and leaves its partial sums there; each call writes
 * every slot it reads before reading it, so nothing is cleared between
 * calls.  Calls that overlap on the GPU (other streams, other host threads)
 * race on the array and must be serialised by the caller.  Returns
 * DSO_EINVAL for bad arguments and DSO_ECUDA for CUDA errors; it does not
 * set the text returned by dso_last_error. */
dso_status dso_position_observables_noalloc(const void* psi, const double* V, int S, int64_t P, double dV,
                                            double* out, void* cuda_stream);

/* Diagnostics: the rate (instructions per second, written to *inst_per_s)
 * at which CUDA device `device` retires FP64 fused multiply-adds with all
 * three operands in per-thread registers -- the operand pattern of the FFT
 * butterflies, potential matvecs and kinetic phases of the FP64 path, which
 * is bound by the FP64 pipe.  Runs a short microbenchmark (a few
 * tens of milliseconds) on a stream of its own and synchronises it; the best of three
 * timed launches is reported.  The paper has no counterpart: this is the
 * denominator of the instruction-rate roofline of the FP64 kernels. */
dso_status dso_fp64_issue_rate(int device, double* inst_per_s);

/* Pass limits of a context: an axis longer than max_line points, or an axis
 * 0 whose S surfaces exceed max_tile points, is transformed as two virtual
 * axes (four-step FFT, see dso_set_grid).  Powers of two, max_line in
 * [8, 4096] (default 4096), max_tile in [16, 8192] (default 8192).  Smaller
 * limits give smaller tiles (more of them, for small grids) at the cost of
 * more passes; a grid that no longer fits (a split factor above max_line)
 * returns DSO_EINVAL and keeps the old limits.  Takes effect at once when the
 * potential is loaded (the state is kept), else at dso_load_potential.  A
 * context added to a batch gets the batch's limits (1024, 2048); setting the
 * same limits on a context that propagates alone gives it the batch's pass
 * layout, so that the two give bitwise the same result.  Without this call,
 * a 1-D grid that the default limits keep as one line (S n <= 8192) has its
 * limits chosen by timing a step under a few candidates at its first
 * propagation (one line keeps a small job on one SM; a split spreads it over
 * many), cached for the process per grid, S, precision and elementary method
 * (not per batch size, so a batch and its jobs alone share the layout).  The
 * paper has no counterpart. */
dso_status dso_set_pass_limits(dso_ctx* ctx, int max_line, int max_tile);

/* Step boundaries.  In a symmetric composition the first and last a~
 * coefficients belong to the same operator (the potential for DSO_VTV, the
 * kinetic step for DSO_TVT), so the last action of one time step and the
 * first of the next act back to back and form one action with coefficient
 * a~_last + a~_0, the merge of adjacent actions of Sec. II F applied across
 * the step boundary.  merged = 1 (the default) gives that action a table of
 * its own (one more table when a~_last + a~_0 is not already a unique value)
 * and applies it once; merged = 0 applies the two tables one after the other
 * in one pass.  The two agree to round-off; the first step and the final
 * action of a propagation are not affected.  Any other value returns
 * DSO_EINVAL.  Drops the context's tables and tuning; the state is kept. */
dso_status dso_set_boundary_merge(dso_ctx* ctx, int merged);

/* Form of the kinetic step U_T(dt) = exp(-i dt T(p)) of Sec. II G.  With the
 * diagonal mass matrix of Eq. (diab_mol_ham), T = sum_d p_d^2 / (2 m_d) and
 * the per-axis factors commute, so U_T is the product over the axes of
 * exp(-i dt p_d^2 / (2 m_d)), each diagonal in that axis's own momentum
 * representation.  DSO_KINETIC_JOINT transforms all axes forward, applies
 * the phase of the whole grid and transforms back (four passes per substep
 * on a 3-D grid, one table of P entries per unique kinetic coefficient).
 * DSO_KINETIC_AXES applies each axis's phase between that axis's own forward
 * and inverse FFT, in one pass per axis with the potential step joined to
 * the axis-0 pass (three passes per substep on a 3-D grid, tables of
 * n_0 + .. + n_{D-1} entries, D - 1 more phase multiplications per
 * amplitude); the result agrees with the joint form to round-off.
 * DSO_KINETIC_AUTO (the default) takes the per-axis form in DSO_FP32 mode,
 * whose passes are bound by memory traffic (one wavefunction round trip per
 * substep fewer), and the joint form in DSO_FP64 mode, whose passes are bound
 * by FP64 arithmetic.  Grids with one axis, or with an axis split into two
 * virtual axes (dso_set_pass_limits), always use the joint form.  Any other
 * mode returns DSO_EINVAL.  Drops the context's tables and tuning; the state
 * is kept. */
dso_status dso_set_kinetic_mode(dso_ctx* ctx, int mode);

/* Plane pass of the kinetic step on 3-D grids.  The kinetic step's work on
 * the two last axes d = 1, 2 takes one round trip of the wavefunction
 * through device memory per pass: with the per-axis step (dso_set_kinetic_
 * mode) [F1 T1 I1] [F2 T2 I2], with the joint step [F1] [F2 T I2] [I1].  The
 * plane pass runs them in one launch: each n_1 x n_2 plane of one surface is
 * held by one cluster of CTAs, which transforms its columns, exchanges the
 * plane through the CTAs' shared memory and transforms its rows (per axis:
 * each axis's phase between its own FFTs; joint: the grid's phase between
 * the row FFTs, then a second exchange and the inverse column FFTs).  The
 * same FFTs, phases and products in the same order: the result is bitwise
 * that of the line passes.  Applies to 3-D grids of whole axes (none split)
 * with n_1 and n_2 in {32, 64, 128}; elsewhere, and for jobs in a batch
 * slot, the mode has no effect.  DSO_PLANE_ON uses it
 * wherever it applies; DSO_PLANE_OFF never; DSO_PLANE_AUTO (the default)
 * lets the autotuner time a middle step both ways and keep the faster (with
 * autotuning off, as DSO_PLANE_OFF).  Any other mode returns DSO_EINVAL.
 * Drops the context's tuning; the state and tables are kept. */
dso_status dso_set_plane_pass(dso_ctx* ctx, int mode);

/* Potential operators precomputed or built per action (Sec. II F's
 * memory/time trade-off).  DSO_OPERATORS_TABLES precomputes U_a(q) =
 * exp(-i a dt V(q)) for every unique potential coefficient a (S(S+1)/2
 * complex entries per grid point and coefficient, per job).
 * DSO_OPERATORS_ON_THE_FLY stores, per grid point, only the part of U that
 * does not depend on the coefficient -- for S = 2 the mean, half difference
 * and coupling of V and its rotation rate (4 doubles), for S >= 3 the
 * eigenvectors and eigenvalues of V (S^2 + S doubles) -- and assembles the
 * table of each potential action into one of two slots right before the
 * pass that applies it: one more kernel per action, table memory
 * independent of the number of unique coefficients, and bitwise the same
 * propagation.  DSO_OPERATORS_AUTO (the default) precomputes the tables when
 * they take at most half the device memory free when the tables are built,
 * and builds per action otherwise.  The kinetic tables are always
 * precomputed (one phase per grid point, or per axis point, per coefficient).
 * Jobs in a batch slot always use precomputed tables
 * (DSO_OPERATORS_ON_THE_FLY makes dso_batch_add return DSO_EINVAL).  Any
 * other mode returns DSO_EINVAL.  Drops the context's tables and tuning; the
 * state is kept. */
dso_status dso_set_operator_mode(dso_ctx* ctx, int mode);

/* 1 when the context's current tables build the potential operators per
 * action, 0 when they are precomputed (or not built yet); DSO_EINVAL for a
 * null context. */
int dso_operators_on_the_fly(const dso_ctx* ctx);

/* Batch slots (continuous batching).  A batch advances many jobs -- each a
 * context with its own grid, surfaces, masses, potential, scheme and state,
 * all of the batch's precision and device -- by one composed time step of
 * each job per launch of one persistent kernel: the launch's work list holds
 * every pass of every unfinished job (tiles of one pass of one job wait for
 * the job's previous pass through a counter; the waits are bounded).  Jobs
 * with uneven grids and different schemes, time steps and step counts share
 * the launch; jobs join (dso_batch_add) and leave (dso_batch_retire) between
 * steps.  Each job's result is bitwise the same as the job propagated alone
 * with the batch's pass limits (dso_set_pass_limits(ctx, 1024, 2048)), and
 * so within round-off of the job alone with the defaults.
 *
 * dso_batch_create: an empty batch on `device`, with precision DSO_FP64 or
 * DSO_FP32, working on `cuda_stream` (NULL: a stream the batch owns).
 * dso_batch_destroy: releases the batch; the jobs' contexts stay the
 * caller's. */
typedef struct dso_batch dso_batch;
dso_status dso_batch_create(dso_batch** out, int device, int precision, void* cuda_stream);
void dso_batch_destroy(dso_batch* batch);

/* Add a ready context (grid, masses, potential, scheme and psi set) as a job
 * that is to advance its psi by time t with step dt (t/dt a non-negative
 * integer within 1e-9 relative, dt may be negative), as dso_propagate(ctx, t,
 * dt) would.  The context is borrowed until dso_batch_retire: the caller must
 * not use it meanwhile.  Its tables are built for dt and its passes re-planned
 * with the batch's limits; *slot receives the job's slot.  DSO_EINVAL for a
 * grid too large for a slot (lines above 1024 points after one split, or
 * S x n1 above 2048 on axis 0): such a job fills the GPU alone. */
dso_status dso_batch_add(dso_batch* batch, dso_ctx* job, double t, double dt, int* slot);

/* Enqueue one composed step of every unfinished job (its first step's passes
 * the first time, the final pass after its last step): one launch of the
 * work-list kernel, asynchronous on the batch's stream.  *active (may be
 * NULL) receives the number of jobs still unfinished after this step.  Waits
 * for the previous launch before reusing its host-side list. */
dso_status dso_batch_step(dso_batch* batch, int* active);

/* Wait for the batch's work and report a bounded wait that gave up
 * (DSO_ETIMEOUT). */
dso_status dso_batch_sync(dso_batch* batch);

/* Steps done and steps in all of the job in `slot`. */
dso_status dso_batch_slot_status(const dso_batch* batch, int slot, int64_t* steps_done, int64_t* steps_total);

/* Remove the job in `slot` (finished or not) and hand its context back to
 * the caller, whose psi then holds the job's state (synchronises the batch's
 * stream).  The slot is free for a later dso_batch_add. */
dso_status dso_batch_retire(dso_batch* batch, int slot);

/* Launches of the work-list kernel this batch has issued. */
int64_t dso_batch_launch_count(const dso_batch* batch);

/* Non-blocking: 1 while the batch's launched work is pending, 0 when it has
 * finished, a negative dso_status on error (as dso_busy). */
int dso_batch_busy(const dso_batch* batch);

/* Message for the last failed call on this thread (never NULL; valid until
 * the next call on this thread). */
const char* dso_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DSO_H */
