/* GB300-native wall-modelled lattice Boltzmann LES: C ABI of liblbm.so.
 *
 * The library advances a lattice Boltzmann (LB) flow on one CUDA device with one fused
 * collide-and-stream kernel pass per time step. Method (Kummerländer et al., "Large-Scale
 * Simulations of Turbulent Flows using Lattice Boltzmann Methods on Heterogeneous High Performance
 * Computers"):
 *   - homogenised LB update, Eq. (hlbm): f_i(x + c_i, t + 1) = f_i^eq(rho, u_hat)
 *     + (1 - 1/tau_eff) f~_i^(1), read for BGK as f~^(1) = f - f^eq(rho, u) (Sec. 2.2);
 *   - homogenised velocity, Eq. (convexVelocity): u_hat = gamma u + (1 - gamma) u^B, with the
 *     per-cell porosity gamma = 1 - d (1 = fluid);
 *   - Smagorinsky effective relaxation time, Eq. (tauEff) with Eqs. (sgsStress),(turbVisc):
 *     tau_eff = (tau0 + sqrt(tau0^2 + 18 sqrt(2) C_S^2 |Pi^neq| / rho)) / 2;
 *   - Spalding wall function, Eq. (spaldingfunct), on cells next to solids (Sec. 2.2.1): solid
 *     velocity u^B from the wall law and the sigma = 0 finite-difference non-equilibrium part;
 *   - regularised velocity inlet (Sec. 2.2.2), fixed-pressure outlet and full-slip faces (Sec. 3.2),
 *     half-way bounce-back on solid cells;
 *   - body force through the exact-difference shift u_hat += F/rho.
 *
 * Conventions.
 *   Cell index n = x + nx*(y + ny*z), N = nx*ny*nz. Populations i = 0..q-1 in the order
 *   D3Q19: 0 rest; 1..9 = (1,0,0),(0,1,0),(0,0,1),(1,1,0),(1,-1,0),(1,0,1),(1,0,-1),(0,1,1),(0,1,-1);
 *          10..18 their opposites in the same order.
 *   D3Q27: 0 rest; 1..13 = the nine D3Q19 speeds followed by (1,1,1),(1,1,-1),(1,-1,1),(1,-1,-1);
 *          14..26 their opposites.
 *   Population arrays f[i*N + n]; velocity arrays u[a*N + n] (a = 0,1,2 for x,y,z); inlet velocity
 *   uin[a*ny*nz + y + ny*z]. Lattice units: dx = dt = 1, cs^2 = 1/3, nu = (tau - 1/2)/3.
 *   Faces in the order x-, x+, y-, y+, z-, z+.
 *
 * Memory. The context owns every device buffer it allocates (cudaMalloc on the current device at
 * lbm_create) and frees them in lbm_destroy. Caller buffers are never retained after a call returns.
 * Array arguments may be host or device pointers (detected with cudaPointerGetAttributes); a call
 * that reads or writes host memory synchronises the context's stream before it returns, a call on
 * device memory is ordered on that stream. Page-locked (pinned) host fields given to
 * lbm_init_equilibrium and lbm_moments are read and written by the kernels in place over the
 * CPU-GPU link; other host memory is staged through device memory.
 *
 * Errors. Every int-returning call returns LBM_OK or an error code and leaves a message for
 * lbm_last_error() (thread-local). Invalid sizes, codes or pointers give LBM_EINVAL and change
 * nothing. Device-side problems (a non-finite density or momentum seen by a step, an invalid mask
 * code in device memory) set a sticky status word on the device; it is read back by synchronising
 * calls (lbm_sync, lbm_moments, lbm_reduce, ...) which then return LBM_ENAN / LBM_EINVAL.
 */
#ifndef LBM_H_
#define LBM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

enum { LBM_D3Q19 = 19, LBM_D3Q27 = 27 };
/* Population storage. Arithmetic is FP32 for LBM_F32/F16/BF16 and FP64 for LBM_F64. Every form
 * stores the deviation f_i - w_i from the rest-state weights; LBM_F16/LBM_BF16 round it to
 * nearest-even on each store. */
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2, LBM_BF16 = 3 };
enum { LBM_OK = 0, LBM_EINVAL = 1, LBM_ENOMEM = 2, LBM_ECUDA = 3, LBM_ENAN = 4, LBM_ETIMEOUT = 5, LBM_ESTATE = 6 };
/* Mask codes accepted by lbm_set_geometry. */
enum { LBM_CELL_FLUID = 0, LBM_CELL_SOLID = 1, LBM_CELL_INFLOW = 3, LBM_CELL_OUTFLOW = 4 };
/* Classified kinds (low 3 bits of the type byte, see lbm_debug_dump). WALL = non-solid cell with a
 * solid neighbour (or a neighbour beyond a bounce-back face); precedence
 * SOLID > INFLOW > OUTFLOW > WALL > FLUID. */
enum { LBM_KIND_FLUID = 0, LBM_KIND_SOLID = 1, LBM_KIND_WALL = 2, LBM_KIND_INFLOW = 3, LBM_KIND_OUTFLOW = 4 };
/* Face kinds. PERIODIC faces come in pairs. WALL: half-way bounce-back, counts as a solid layer
 * beyond the face. SLIP: specular reflection (Sec. 3.2 full slip). OPEN: populations entering
 * through the face are the unknowns of the INFLOW/OUTFLOW cells on it. */
enum { LBM_FACE_PERIODIC = 0, LBM_FACE_WALL = 1, LBM_FACE_SLIP = 2, LBM_FACE_OPEN = 3 };
/* dtype codes of host/device array arguments of the *_ex calls. */
enum { LBM_DTYPE_F32 = 1, LBM_DTYPE_F64 = 0 };
/* Collision models (lbm_set_collision). */
enum { LBM_BGK = 0, LBM_HRR = 1 };

/* Create a lattice of nx*ny*nz cells with molecular relaxation time tau (> 1/2) and Smagorinsky
 * constant c_smag >= 0 (C_S of Eq. turbVisc; 0 gives plain BGK). Storage LBM_F32, all faces
 * periodic, all cells fluid at rest (f = w). Returns NULL on error (lbm_last_error). */
lbm_ctx* lbm_create(int lattice, int nx, int ny, int nz, double tau, double c_smag);
void lbm_destroy(lbm_ctx* ctx);
const char* lbm_last_error(void);

/* Population storage form; reallocates and resets the state to rest. */
int lbm_set_precision(lbm_ctx* ctx, int storage);
/* Face kinds: px/py/pz != 0 makes both faces of that axis periodic, 0 makes them bounce-back. */
int lbm_set_periodic(lbm_ctx* ctx, int px, int py, int pz);
/* Face kinds, six entries in the order x-, x+, y-, y+, z-, z+ (periodic ones must pair). */
int lbm_set_faces(lbm_ctx* ctx, const int kinds[6]);
/* Geometry: mask (N bytes, codes LBM_CELL_*), wall_dist (N floats, distance of a WALL cell centre
 * from the wall, nullable = 0.5). Runs the classification and builds the boundary-cell list
 * (WALL, INFLOW, OUTFLOW and wall-model reference cells, ascending cell index). Resets to rest. */
int lbm_set_geometry(lbm_ctx* ctx, const uint8_t* mask, const float* wall_dist);
/* Body force per unit volume (lattice units). */
int lbm_set_force(lbm_ctx* ctx, double fx, double fy, double fz);
/* Inlet velocity of INFLOW cells, 3*ny*nz values (inward normal +x). */
int lbm_set_inflow(lbm_ctx* ctx, const float* u_in);
int lbm_set_inflow_ex(lbm_ctx* ctx, const void* u_in, int dtype);
/* Vortex-method turbulent inlet (Sec. 2.2.2). Before every step, n seed points are drawn uniformly
 * on the inlet plane (counter-based SplitMix64 random numbers keyed by seed and the step counter,
 * so a run is reproducible step by step); vortex i has circulation
 * Gamma_i = 4 s_i sqrt(pi k_i A / ((6 ln 3 - 9 ln 2) n)), k_i = 3/2 (|u_mean(p_i)| intensity)^2,
 * A = number of INFLOW cells, random sign s_i; the inlet velocity of the step is the mean profile of
 * lbm_set_inflow plus the in-plane vortex field (profile (1 - e^-a) e^-a / r^2, a = r^2/(2 sigma^2))
 * plus the streamwise fluctuation -(u_v . grad U)/|grad U| with U the streamwise inlet velocity of
 * the previous step. n = 0 switches it off. The inlet field restarts from the mean profile on
 * lbm_set_inflow, lbm_set_vortex_inlet and every state (re)initialisation, and is part of lbm_save.
 * The adjoint calls return LBM_ESTATE while it is on. Errors: LBM_EINVAL for n outside [0, 2^20],
 * sigma <= 0 or intensity < 0. Device memory: 2 * 3 * ny * nz + 3 * n compute-type values. */
int lbm_set_vortex_inlet(lbm_ctx* ctx, int n, double sigma, double intensity, unsigned long long seed);
/* Outlet density of OUTFLOW cells (inward normal -x). */
int lbm_set_outflow(lbm_ctx* ctx, double rho_out);
/* Outlet fringe zone (Sec. 3.2: the fixed-pressure outlet has a fringe zone in front of it; the
 * paper gives no parameters, so this layer is a reading). In the last L planes x >= nx - L, every
 * cell that is neither INFLOW nor OUTFLOW relaxes its post-collision populations towards the
 * equilibrium at the outlet density (lbm_set_outflow) and its own reported velocity u:
 *   f*_i <- f*_i - s(x) (f*_i - f^eq_i(rho_out, u)),  s(x) = s_max xi^p,  xi = (x - (nx - L) + 1) / L,
 * so s rises from s_max L^-p at the first plane of the layer to s_max at x = nx - 1 (p = 0: constant).
 * L = 0 switches it off. The adjoint calls return LBM_ESTATE while it is on. Errors: LBM_EINVAL for L
 * outside [0, nx], s_max outside [0, 1] or p < 0. Device memory: nx compute-type values. */
int lbm_set_fringe(lbm_ctx* ctx, int L, double s_max, double p);
/* Slab sub-domain of a z decomposition (the paper's domain decomposition, Sec. 3.1, cut along the
 * slowest axis). The first lo and last hi z-planes (0 or 2 each) are ghost planes: they hold the
 * neighbouring sub-domains' cells (their mask, wall distance, porosity, inlet velocity and initial
 * state, passed like every other cell), are classified like every cell and are never updated. The
 * real cells then step exactly as in the whole domain provided the caller runs the halo exchange
 * below around every step. Rebuilds the geometry and resets the state to rest. The BGK collision
 * with a steady inlet only (LBM_ESTATE for LBM_HRR, the vortex inlet and the adjoint calls).
 * Errors: LBM_EINVAL for lo or hi not 0 or 2, or lo + hi >= nz. */
int lbm_set_ghost_planes(lbm_ctx* ctx, int lo, int hi);
/* Halo lists of side 0 (the z- cut) and side 1 (the z+ cut). With zr the real boundary plane and zg
 * the adjacent ghost plane, entries run over the plane positions pos = x + nx*y ascending, then the
 * population slots p ascending:
 *   list 0: the slots of zr cells that non-solid cells of zg read and write in an odd step (their
 *           streaming, bounce-back and slip rules): the post-collision populations opp(p) that leave
 *           through the cut;
 *   list 1: the slots of zg cells that non-solid cells of zr read and write in an odd step;
 *   list 2: the zr cells that a WALL cell of zg takes as wall-model reference cell;
 *   list 3: the zg cells that a WALL cell of zr takes as reference cell.
 * Populations travel as stored (storage type, deviations f - w, one value per entry), reference
 * velocities as 3 compute-type values per entry. The neighbour's list 1 (3) on the other side of the
 * same cut equals this list 0 (2) entry by entry. Exchange schedule (in-place streaming: even steps
 * touch only a cell's own slots), for both sides:
 *   before a step that starts at an odd step count: pack list 0, send it; unpack the neighbour's into
 *   list 1; after that step: pack list 1, send it; unpack the neighbour's into list 0;
 *   after every step: pack list 2, send it; unpack the neighbour's into list 3.
 * After an odd number of steps the state is stored swapped (a cell's incoming populations sit in its
 * neighbours' slots), so reading it (lbm_moments, lbm_get_populations, lbm_reduce) needs the ghost
 * slots current: run the list 0 -> list 1 exchange of the coming odd step first (it need not be
 * repeated before that step).
 * lbm_halo_count gives the number of entries; pack (lists 0, 1, 2) and unpack (lists 0, 1, 3) take a
 * host or device buffer of the context's device (device buffers: ordered on the context stream;
 * host buffers: the call synchronises). The lists are also readable through lbm_debug_dump. */
int lbm_halo_count(lbm_ctx* ctx, int side, int list, int64_t* n);
int lbm_halo_pack(lbm_ctx* ctx, int side, int list, void* buf);
int lbm_halo_unpack(lbm_ctx* ctx, int side, int list, const void* buf);
/* Per-cell porosity gamma (N values in [0,1], 1 = fluid); NULL removes it. */
int lbm_set_porosity(lbm_ctx* ctx, const float* gamma);
int lbm_set_porosity_ex(lbm_ctx* ctx, const void* gamma, int dtype);
/* Porosity from a per-cell permeability K (N values, lattice units K/dx^2; +inf = fluid; K <= 0 or
 * NaN = impermeable): the
 * lattice porosity of Eq. lattice_porosity, gamma = 1 - nu tau / K with nu = (tau - 1/2)/3 and tau
 * the molecular relaxation time, read as the fluid fraction and clamped to [0, 1]; replaces any
 * porosity set before. Errors: LBM_EINVAL for a bad pointer or dtype. */
int lbm_set_permeability(lbm_ctx* ctx, const float* K);
int lbm_set_permeability_ex(lbm_ctx* ctx, const void* K, int dtype);
/* Forchheimer permeability of a sample (Sec. 2.1): K = mu Q / (A (dP/L - rho Q^2 / (K_beta A^2))),
 * K_beta = +inf for Darcy's law. Any consistent units; NaN when the bracket is not positive or
 * A, L <= 0. No context, no device work. */
double lbm_forchheimer_permeability(double mu, double Q, double A, double L, double dP, double rho, double K_beta);
/* Spalding wall function on WALL cells with von Karman constant kappa and wall constant E
 * (kappa <= 0 switches it off: WALL cells then collide like fluid cells with bounce-back). */
int lbm_set_wall_model(lbm_ctx* ctx, double kappa, double E);
/* Collision model (Sec. 2.2, Eq. hlbm). LBM_BGK (default): f^(1) = f - f^eq(rho, u), second-order
 * equilibrium. LBM_HRR: the hybrid recursive regularised form: third-order Hermite equilibrium,
 * f^(1) rebuilt from the second-order coefficient A2 = sigma Pi^neq + (1 - sigma) Pi^FD and its
 * recursive third-order extension, Pi^FD = -2 rho cs^2 tau S^FD with S^FD the central-difference
 * strain of the previous step's velocity field (one-sided next to solids and non-periodic faces);
 * WALL cells with the wall model use sigma = 0 with the modelled strain. sigma in [0, 1]; 1 needs no
 * velocity field. The HRR form keeps a velocity field of 3*N compute-type values (two copies,
 * allocated here, released on LBM_BGK); it is rebuilt from the state before the first step after
 * any state change and is part of lbm_save. The adjoint calls return LBM_ESTATE under LBM_HRR.
 * Errors: LBM_EINVAL for an unknown model or sigma outside [0, 1]. */
int lbm_set_collision(lbm_ctx* ctx, int model, double sigma);
/* Equilibrium state f_i = f_i^eq(rho, u) (rho: N values, u: 3*N values); step counter to 0; the
 * wall-model reference buffer is filled with this state's velocity. */
int lbm_init_equilibrium(lbm_ctx* ctx, const float* rho, const float* u);
int lbm_init_equilibrium_ex(lbm_ctx* ctx, const void* rho, const void* u, int dtype);

/* Advance n time steps (stream-ordered, asynchronous). Returns the sticky status seen so far. */
int lbm_step(lbm_ctx* ctx, int n);
/* Same (n >= 1), timed with CUDA events on the context stream: adds the device time of the
 * interior-cell kernels to ms[0], of the rest of each step (wall-model pass, boundary-list kernel)
 * to ms[1], and the time from the first step's start to the last step's end to ms[2]. Synchronises. */
int lbm_step_timed(lbm_ctx* ctx, int n, double ms[3]);
/* Wait for the context stream; returns LBM_ENAN if a step has seen a non-finite density. */
int lbm_sync(lbm_ctx* ctx);

/* Macroscopic fields of the current (pre-collision) state: rho (N), u (3*N) with
 * u = j/rho + F/(2 rho); INFLOW/OUTFLOW cells report their reconstructed state; SOLID cells 0. */
int lbm_moments(lbm_ctx* ctx, float* rho, float* u);
int lbm_moments_ex(lbm_ctx* ctx, void* rho, void* u, int dtype);
/* FP64 reductions over non-solid cells: mass = sum rho, mom = sum rho u. */
int lbm_reduce(lbm_ctx* ctx, double* mass, double mom[3]);
/* Populations f_i (not deviations) of the current state, q*N values. */
int lbm_get_populations(lbm_ctx* ctx, void* f, int dtype);
/* Replace the state by the given populations (q*N values, natural layout); refreshes the
 * wall-model reference buffer from it. */
int lbm_set_populations(lbm_ctx* ctx, const void* f, int dtype);

/* Discrete adjoint (differentiation extension; the paper cites OpenLB as differentiable, Sec. 1).
 * Objective: J = (1/W) sum over the last W of T steps of cs^2 (<rho>_{x=xa} - <rho>_{x=xb}),
 * plane means over non-solid cells of the state after each step.
 * lbm_objective_forward runs T steps from the current state, keeping a copy of the state every
 * ckpt steps (ckpt even), and returns J. lbm_objective_backward then recomputes each segment from
 * its checkpoint into a ring of states and sweeps the adjoint kernel backwards. ckpt = 1 (T even)
 * keeps every state instead, (T + 1) * q * N storage values in device memory (LBM_ENOMEM if they do
 * not fit; they stay allocated until the next forward run or lbm_destroy): the forward steps out of
 * place from each state into the next, and the backward is the reverse sweep alone. Both accumulate
 * dJ/dgamma and dJ/du_in over all T steps in FP64 device arrays (whatever the storage), and writes
 * them to dJ_dgamma (N doubles) and dJ_duin (3*ny*nz doubles), host memory or device memory of the
 * context's device; either may be NULL. The wall model is not differentiated (LBM_ESTATE if it is
 * on). After backward the state is the one at the end of the forward run. */
int lbm_objective_forward(lbm_ctx* ctx, int T, int W, int xa, int xb, int ckpt, double* J);
int lbm_objective_backward(lbm_ctx* ctx, double* dJ_dgamma, double* dJ_duin);
/* One reverse step at the current state: lam_out = (dS_{t+1}/dS_t)^T lam_in (q*N values each,
 * natural layout, dtype LBM_DTYPE_*), and writes (dS_{t+1}/dgamma)^T lam_in to dgamma (N, FP64) and
 * (dS_{t+1}/du_in)^T lam_in to duin (3*ny*nz, FP64); both nullable; host or device memory. This is
 * the single-step building block (the vector-Jacobian product of one step); the whole-run gradient
 * with checkpointing is lbm_objective_forward/backward. */
int lbm_adjoint_step(lbm_ctx* ctx, const void* lam_in, void* lam_out, int dtype, double* dgamma, double* duin);
/* Device times (CUDA events) of the last differentiation run: ms[0] segment recomputation and
 * ms[1] reverse sweep of lbm_objective_backward, ms[2] the whole lbm_objective_forward. */
int lbm_adjoint_timing(lbm_ctx* ctx, double ms[3]);

/* Checkpoint of the whole state (populations, step counter, reference buffer). With buf == NULL,
 * *len receives the size needed. lbm_load restores a buffer written by lbm_save of a context with
 * the same lattice, size, storage and geometry. */
int lbm_save(lbm_ctx* ctx, void* buf, size_t* len);
int lbm_load(lbm_ctx* ctx, const void* buf, size_t len);

/* Stream for all work of the context (e.g. torch.cuda.current_stream().cuda_stream); 0 = default. */
int lbm_set_stream(lbm_ctx* ctx, void* cuda_stream);

/* Options. LBM_OPT_KERNEL: 0 (default) runs interior cells with the plain kernel (one thread per
 * cell, direct coalesced loads and stores); 2 runs them with the shared-memory staged kernel (bulk
 * asynchronous copies of 128-cell x-segments) when nx is a multiple of 128 and the storage is not
 * LBM_F64, else the plain one. LBM_OPT_DEBUG_STALL: 1 makes the staged kernel also wait on a
 * barrier that nothing completes, so that its bounded wait (one second) runs out: the step then
 * ends early, the status word records it and the next synchronising call returns LBM_ETIMEOUT
 * (the state must be re-initialised); used to test that path without a GPU fault. */
enum { LBM_OPT_KERNEL = 1, LBM_OPT_DEBUG_STALL = 2 };
int lbm_set_option(lbm_ctx* ctx, int option, int value);

/* Counters: out[0] N, [1] boundary-list length, [2] WALL, [3] reference cells, [4] INFLOW,
 * [5] OUTFLOW, [6] SOLID, [7] steps done, [8] storage, [9] lattice q. */
int lbm_info(lbm_ctx* ctx, int64_t out[10]);
/* Interior kernel the next step runs: 0 one cell per thread, 1 cell pairs (two cells per thread with
 * packed FP32 arithmetic, FP32 or 16-bit storage, when at most 2 % of the 64-cell x-groups would mix
 * pairs of plain cells with pairs on the per-cell path; nx even, indices within 32 bits), 2 the
 * staged kernel (LBM_OPT_KERNEL = 2), 3 four cells per thread on even steps and cell pairs on odd
 * steps (where 1 would be chosen, for D3Q19 BGK with FP16 or BF16 storage and nx a multiple of 4).
 * Negative on a null context. */
int lbm_interior_kernel(lbm_ctx* ctx);
/* Number of kernels the step calls (lbm_step, lbm_step_timed) of this context have launched so far:
 * per step the wall-model state pass (when the wall model is on and WALL cells are handled inline),
 * the interior kernel, the boundary-list kernel (when list cells remain for it), and the vortex-inlet
 * and velocity-field kernels when those forms are on. */
int lbm_launch_count(lbm_ctx* ctx, int64_t* n);
/* Integer maps for bit-exact tests: which = 0 type byte per cell (N; bits 0-2 kind, bit 3
 * reference cell, bit 4 a source position is solid or outside, bit 5 boundary list, bit 7 ghost
 * plane of a slab sub-domain, bit 6 list cell
 * updated by the interior kernel: INFLOW/OUTFLOW cells, and WALL/reference cells in 32-cell
 * x-groups holding >= 8 list cells);
 * 1 boundary-list cells; 2 list position of each entry's reference cell (-1 none);
 * 3 integer wall-normal sums v of each entry (3 per entry, sum of W_i c_i over solid neighbours,
 * W_i = 36 w_i for D3Q19 and 216 w_i for D3Q27); 4 source population j and 5 source cell m of each
 * (i, n) (q*N each, i-major; f_i(n, t+1) = f*_j(m, t); -1 for solid cells); 6..13 the halo list
 * (which - 6) % 4 of side (which - 6) / 4 of a slab sub-domain (lbm_halo_count entries: p*nx*ny + pos
 * for lists 0 and 1, pos for lists 2 and 3). */
int lbm_debug_dump(lbm_ctx* ctx, int which, int64_t* out, size_t count);

/* Allocation-free reduction (no counterpart in the paper: an addition for callers of this library).
 * Some callers cannot let a library allocate device memory: applications whose pool allocator owns
 * all device memory, codes running at the memory limit, loops that must not pay for an allocation
 * between steps. lbm_reduce_static serves them: it sums mass = sum_i f_i and momentum
 * sum_i f_i c_i over the cells of a caller-owned population array, keeping its partial sums in a
 * fixed static device array (4 doubles per 65536 cells, 128 KiB, held by every GPU that loads the
 * library until the process exits) and calling no cudaMalloc, cudaFree or allocating routine.
 *   lattice: 19 or 27 (velocity order as above); f: q*n_cells values of dtype (LBM_DTYPE_F32 or
 *   LBM_DTYPE_F64), f[i*n_cells + n] (populations, not deviations), device or managed memory of the
 *   current device; mask: n_cells mask bytes in device or managed memory of the current device
 *   (cells with code LBM_CELL_SOLID are skipped) or NULL;
 *   n_cells: 1..LBM_REDUCE_STATIC_MAX_CELLS, larger sizes are rejected with LBM_EINVAL;
 *   out: 4 doubles (mass, momentum x, y, z), device or managed memory of the current device (written
 *   on the stream) or host memory (the call then synchronises the stream); stream: cudaStream_t or
 *   NULL for the default stream. A pointer of the wrong kind or on another device gives LBM_EINVAL
 *   before any work is queued.
 * The first call made on a device looks up the static array's device address (make that first
 * call before any stream capture); the address stays cached for the process, so the call must not
 * be used on a device after a cudaDeviceReset of it. All calls share the array, so calls that
 * overlap on the GPU race; each call overwrites the partial sums it reads. Errors: LBM_EINVAL
 * (arguments), LBM_ECUDA; message in lbm_reduce_static_error(). */
#define LBM_REDUCE_STATIC_MAX_CELLS 268435456LL
int lbm_reduce_static(int lattice, const void* f, int dtype, const uint8_t* mask, int64_t n_cells, double* out,
                      void* stream);
const char* lbm_reduce_static_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H_ */
