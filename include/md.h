/*
 * md.h -- C ABI of the GB300 many-body molecular-dynamics library (libmd.so).
 *
 * The library evaluates the per-step hot path of molecular dynamics with
 * embedded-atom / second-moment tight-binding potentials as described by
 * Hou et al., "Molecular dynamics simulations with many-body potentials on
 * multiple GPUs" (arXiv:1212.6332):
 *   - cell binning and a Verlet neighbour list            (Sec. 3.2, Fig. 3)
 *   - the density pass rho_i = sum_j rho(r_ij)            (Sec. 3.3, Fig. 5)
 *   - the embedding derivative F'(rho_i)                  (Eq. 3)
 *   - the force pass of Eq. (3)                           (Sec. 3.3, Fig. 6)
 *   - time integration (velocity Verlet here; the paper uses a
 *     predictor-corrector, Sec. 3.3)
 *   - many independent boxes in one run                   (Sec. 4.4)
 * plus parameter gradients of a force-matching loss (no counterpart in the
 * paper).
 *
 * Conventions for every entry point:
 *   - Units: Angstrom, eV, fs, atomic mass unit (u), kelvin.
 *   - Atom arrays are in the caller's atom order, row-major [n_atoms][3]
 *     float64 for 3-vectors. Internally atoms are re-sorted by cell; the
 *     library maps back on every input and output.
 *   - Pointer arguments marked "host or device" may point to host memory
 *     (pageable or pinned) or to device memory of the current device; host
 *     memory is copied with cudaMemcpyAsync through a device staging buffer
 *     (pinned memory copies fastest). Pointers
 *     marked "device" must be device memory. The caller owns every pointer
 *     it passes; the library owns its handles and internal buffers and
 *     frees them in md_destroy / md_batch_destroy.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream). Outputs written to device memory are valid once
 *     the stream reaches that point; outputs written to host memory are
 *     valid when the call returns (the call synchronizes the stream).
 *   - Every call returns an md_status. Argument errors are detected on the
 *     host before any work is enqueued. Device-side conditions (neighbour
 *     overflow beyond the regrow cap, non-finite energies) are recorded in
 *     a device status word and returned by the next call that synchronizes.
 *     md_last_error() gives a text for the last failure on a handle;
 *     md_status_string() names a code. No C++ exception crosses the ABI.
 *   - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef MD_H
#define MD_H

#include <stdint.h>

#if defined(__GNUC__)
#define MD_API __attribute__((visibility("default")))
#else
#define MD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* md_stream; /* identical to cudaStream_t */
typedef struct md_batch md_batch;
typedef md_batch md_ctx; /* a single box is a batch of one box */

enum md_status {
    MD_OK = 0,
    MD_ERR_ARG = 1,            /* invalid argument (nothing enqueued) */
    MD_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    MD_ERR_NOMEM = 3,          /* device allocation failed */
    MD_ERR_NEIGH_OVERFLOW = 4, /* neighbour list exceeded the regrow cap */
    MD_ERR_NONFINITE = 5,      /* a non-finite energy or force appeared */
    MD_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
    MD_ERR_UNSUPPORTED = 7     /* valid but not supported combination */
};

enum md_precision {
    MD_FP64 = 0,  /* float64 accuracy: float64 state, pair functions and
                     F'; r^2 and separations exact in fixed point, the
                     density totals exact integer sums, the force sums of
                     Eq. (3) in float32 pieces with float-float totals
                     (about 2^-46 of a term) */
    MD_MIXED = 1  /* float32 pair math relative to cell-local origins;
                     compensated sums; float64 positions, velocities and
                     integration */
};

enum md_pot_kind {
    MD_POT_RGL = 0,   /* second-moment tight binding (Cleri-Rosato):
                         V = 2A exp(-p(r/r0-1)) S(r),
                         rho = xi^2 exp(-2q(r/r0-1)) S(r), F = -sqrt(rho);
                         p[] = {A, xi, p, q, r0} */
    MD_POT_SC = 1,    /* Sutton-Chen: V = eps (a/r)^n S(r),
                         rho = (a/r)^m S(r), F = -c eps sqrt(rho);
                         p[] = {eps, c, a, n, m} */
    MD_POT_SPLINE = 2 /* V, rho natural cubic splines of knot values on a
                         uniform grid over [r_lo, r_hi] (zero for
                         r >= r_hi, linear below r_lo); F a natural cubic
                         spline over [rho_lo, rho_hi], linear outside */
};

/* Potential of Eq. (1): pair term V, density function rho, embedding F.
 * S(r) is the C2 taper 1 - 10x^3 + 15x^4 - 6x^5, x = (r - r_taper) /
 * (r_cut - r_taper), S = 1 below r_taper and 0 from r_cut on; r_taper >=
 * r_cut gives a hard cut. F(rho) = F'(rho) = 0 for rho <= 0 (RGL, SC). */
typedef struct md_potential {
    int kind;              /* enum md_pot_kind */
    double p[8];           /* parameters, see enum md_pot_kind */
    double r_taper, r_cut; /* taper interval (RGL, SC); spline: ignored, r_cut = r_hi */
    const double* knots;   /* spline only: host array of n_phi + n_f + n_F
                              knot values, V knots then rho knots then F knots */
    int n_phi, n_f, n_F;   /* spline knot counts, each >= 4 */
    double r_lo, r_hi;     /* spline V and rho range */
    double rho_lo, rho_hi; /* spline F range */
    int n_types;           /* species (splines only; 0 or 1: one). With T > 1
                              species, Eq. (1)-(3) with type labels: V^(ab)
                              and rho^(ab) per unordered type pair a <= b
                              (symmetric, as the common factor (F'_i + F'_j)
                              of Eq. (3) requires) and F^(a) per type; knots
                              then hold the T(T+1)/2 V tables (pairs in
                              row-major order (0,0), (0,1), ..., (1,1), ...,
                              n_phi values each), the rho tables (n_f each)
                              and the T F tables (n_F each). At most 4. */
} md_potential;

/* Run configuration. box[] is used by md_create only (md_batch_create takes
 * one box per batch member). The neighbour list radius is r_cut + skin; it
 * is rebuilt when some atom has moved more than skin/2 since the last build
 * (Sec. 4.2 uses a list radius beyond the force cutoff). The cells of a box
 * are the largest count per axis with side >= r_cut + skin; every box
 * needs r_cut + skin < L/2 on each axis (minimum image). */
typedef struct md_config {
    double box[3];     /* orthorhombic periodic box lengths, A */
    double skin;       /* neighbour-list skin, A (>= 0) */
    double dt;         /* time step, fs */
    double mass;       /* atomic mass, u (one species) */
    int precision;     /* enum md_precision */
    int max_neighbors; /* initial list capacity per atom; 0 = automatic */
} md_config;

/* Thermodynamic state after the last completed step (or set_state). */
typedef struct md_thermo {
    double ke;          /* kinetic energy, eV: 1/2 sum m v^2 */
    double pe;          /* potential energy E_T of Eq. (2), eV */
    double etot;        /* ke + pe */
    double temperature; /* 2 ke / ((3N - 3) k_B), K; summed over all boxes */
    double max_disp;    /* largest displacement since the last list build, A */
    int64_t n_rebuild;  /* list builds since set_state (excluding its own) */
    int64_t step;       /* steps taken since set_state */
} md_thermo;

/* ---------------------------------------------------------------- single box */

/* Creates a single-box context for n_atoms atoms: the initialisation of
 * Sec. 3.1, which allocates the device arrays of positions, velocities,
 * forces, neighbour counts, the neighbour list with a maximum count per atom
 * (MN there; max_neighbors here, regrown on overflow) and densities, for a
 * system whose energy is Eq. (1)-(2) with the potential `pot` (Sec. 2).
 * Cell tables (Sec. 3.2) are allocated as well. No state is set: call
 * md_set_state or md_compute_forces next. *out receives the handle.
 * Errors: MD_ERR_ARG (bad config or potential, box too small for the list
 * radius), MD_ERR_NOMEM, MD_ERR_CUDA. */
MD_API int md_create(const md_config* cfg, const md_potential* pot, int64_t n_atoms, md_ctx** out);

/* Frees the handle and all the device arrays that md_create allocated
 * (those of Sec. 3.1; the paper does not describe releasing them, so this
 * call has no counterpart in the paper). Synchronizes the device.
 * MD_ERR_ARG for a NULL handle. */
MD_API int md_destroy(md_ctx* ctx);

/* Sets positions x [n][3] and velocities v [n][3] (host or device; v may be
 * NULL for zero velocities): the state of Sec. 2 that Sec. 3.1 copies to the
 * device arrays of positions and velocities. Positions are wrapped into the
 * box (x - L floor(x/L), folded into [0, L)), atoms are
 * binned and sorted, the neighbour list is built and forces are evaluated,
 * so that md_step can start. Resets the step and rebuild counters.
 * Lists built before are kept for positions within half the skin of their
 * build positions (boxes that moved farther are rebuilt). A position equal
 * to the one md_get_state reports for the current state keeps the current
 * one exactly, and when every position does so (a state read back and
 * loaded again, or new velocities only) the current forces are kept too:
 * they are the forces of these positions (not after a step with the
 * pressure coupling of Eq. (5), whose box scaling follows the force pass). */
MD_API int md_set_state(md_ctx* ctx, const double* x, const double* v, md_stream stream);

/* Copies the current positions and/or velocities (either may be NULL) to
 * x, v [n][3] (host or device), caller order: the copy of the device
 * arrays of positions and velocities back to the host of Sec. 3.3 (Fig. 4),
 * mapped back through the cell sort of Sec. 3.2 (the paper's index array
 * from sorted to original atoms). Positions are wrapped into [0, L). */
MD_API int md_get_state(md_ctx* ctx, double* x, double* v, md_stream stream);

/* Rebuilds cells and the neighbour list from the current positions
 * (Sec. 3.2): counting sort of atoms into Morton-ordered cells, then the
 * full list (both i->j and j->i) of pairs with minimum-image
 * r^2 < (r_cut + skin)^2, r^2 = dx*dx + dy*dy + dz*dz evaluated left to
 * right in float64 without fused multiply-add. Grows the list capacity and
 * retries on overflow (up to 4 times; then MD_ERR_NEIGH_OVERFLOW). */
MD_API int md_build_neighbors(md_ctx* ctx, md_stream stream);

/* Copies the current neighbour list of Sec. 3.2 (Fig. 3) in caller ids:
 * nn [n] (device) gets each atom's count, nl [n][ld] (device) its
 * neighbours (unordered; slots
 * beyond the count are left untouched). MD_ERR_ARG if ld is smaller than
 * the largest count (query it with md_max_count). */
MD_API int md_get_neighbors(md_ctx* ctx, int32_t* nn, int32_t* nl, int32_t ld, md_stream stream);

/* Largest neighbour count of the current list (synchronizes): the quantity
 * that bounds MN, the list capacity of Sec. 3.1. */
MD_API int md_max_count(md_ctx* ctx, int32_t* out);

/* Sets positions x [n][3] (host or device; velocities are kept), rebuilds
 * cells and list, runs the density pass (Fig. 5) and force pass (Fig. 6),
 * and writes forces f [n][3] (eV/A), per-atom energies e_atom [n]
 * (E_i of Eq. 1), densities rho [n] and the total energy e_total [1] (E_T
 * of Eq. 2). Every output is optional (NULL) and may be host or device. */
MD_API int md_compute_forces(md_ctx* ctx, const double* x, double* f, double* e_atom, double* rho, double* e_total,
                      md_stream stream);

/* Copies forces f_i of Eq. (3), per-atom energies E_i of Eq. (1) and
 * densities rho_i of Sec. 2 of the current state (each optional; host or
 * device). */
MD_API int md_get_forces(md_ctx* ctx, double* f, double* e_atom, double* rho, md_stream stream);

/* Advances n_steps steps of dt, each the step of Sec. 3.3 (Fig. 4):
 * predict, density pass (Fig. 5), force pass of Eq. (3) (Fig. 6), correct,
 * with velocity Verlet as the predictor and corrector:
 *   v += dt/2 F/m; x += dt v; wrap; rebuild the list (Sec. 3.2) if some
 *   atom moved more than skin/2 since the last build (the paper rebuilds
 *   every ten steps, Sec. 4.3); density pass; force pass; v += dt/2 F/m.
 * The rebuild decision is taken on the device (no host synchronization
 * per step). thermo_hist (optional, host or device) receives n_steps rows
 * of (ke, pe, etot, temperature); out (optional, host) the final state's
 * md_thermo. use_graph != 0 replays the steps from a captured CUDA graph
 * (faster for small systems; same results). Without thermo_hist the
 * float64 path forms the pair energies (sum_j V_ij of Eq. 1) on the last
 * step only: dynamics needs rho_i, F and F' alone, so trajectories are
 * unchanged, and every energy this library reports after the call (out,
 * md_get_thermo, md_get_forces) is that of the final positions. */
MD_API int md_step(md_ctx* ctx, int n_steps, md_thermo* out, double* thermo_hist, int use_graph, md_stream stream);

/* The current md_thermo (host): kinetic energy, E_T of Eq. (2) and the
 * temperature of Sec. 2. Synchronizes the stream. */
MD_API int md_get_thermo(md_ctx* ctx, md_thermo* out, md_stream stream);

/* ---------------------------------------------------------------- batches */

/* Creates a batch of n_boxes independent periodic boxes (Sec. 4.4: the
 * cells of box I are numbered after those of boxes 0..I-1 and only cells
 * of the same box neighbour each other). atom_offsets [n_boxes + 1] (host)
 * are prefix sums of the per-box atom counts; box_lengths [n_boxes][3]
 * (host). cfg->box is ignored. */
MD_API int md_batch_create(const md_config* cfg, const md_potential* pot, int n_boxes, const int64_t* atom_offsets,
                    const double* box_lengths, md_batch** out);

/* Frees a batch and its device arrays (no counterpart in the paper, as
 * md_destroy). MD_ERR_ARG for a NULL handle. */
MD_API int md_batch_destroy(md_batch* b);

/* As md_set_state, md_get_state and md_compute_forces, over all boxes back
 * to back (the combined boxes of Sec. 4.4; each box keeps its own periodic
 * images). e_box [n_boxes] (optional, host or device) gets each box's E_T
 * of Eq. (2). */
MD_API int md_batch_set_state(md_batch* b, const double* x, const double* v, md_stream stream);
MD_API int md_batch_get_state(md_batch* b, double* x, double* v, md_stream stream);
MD_API int md_batch_compute_forces(md_batch* b, const double* x, double* f, double* e_box, md_stream stream);

/* Schedules for md_batch_step. */
enum md_schedule {
    MD_SCHED_AUTO = 0, /* the autotuner's choice: the first call of >= 8 steps times 4
                          steps of each schedule (they give the same bits) and keeps
                          the faster for this handle */
    MD_SCHED_BOX = 1,  /* one persistent thread block owns a whole box for all
                          n_steps, positions held in shared memory */
    MD_SCHED_TILE = 2  /* one launch per phase over the atoms of all boxes */
};

/* Advances every box by n_steps steps of Sec. 3.3 (as md_step): the
 * multiple-box-in-one-run scheme of Sec. 4.4 (Table 1), all boxes in one
 * run, with cells numbered box after box and neighbour cells only inside
 * their own box. The state comes from md_batch_set_state and stays on the
 * device between calls (there is no x, v argument).
 * thermo_box [n_boxes][4] (optional, host or device) gets each box's final
 * (ke, pe, etot, temperature). */
MD_API int md_batch_step(md_batch* b, int n_steps, int schedule, int use_graph, double* thermo_box, md_stream stream);

/* The schedule (no counterpart in the paper, which has one: the tile
 * form of Sec. 4.4) the autotuner picked for this batch (MD_SCHED_TILE or
 * MD_SCHED_BOX; 0 before the first MD_SCHED_AUTO call that ran >= 8 steps)
 * and the per-step times it measured, ms. Any output may be NULL. */
MD_API int md_batch_schedule(const md_batch* b, int* choice, double* ms_tile, double* ms_box);

/* Per-box (ke, pe, etot, temperature) of the current state into
 * thermo_box [n_boxes][4] (host or device); pe is E_T of Eq. (2) per box. */
MD_API int md_batch_thermo(md_batch* b, double* thermo_box, md_stream stream);

/* Replaces the parameters of the potential of Eq. (1) (Sec. 2; same kind
 * and knot counts) and re-evaluates forces at the current positions (no
 * list rebuild; the cutoff may not grow). This is how a fitting loop sets
 * theta before md_param_grad. */
MD_API int md_batch_set_potential(md_batch* b, const md_potential* pot, md_stream stream);

/* Temperature control of Sec. 2, Eq. (4) (Finnis et al.): every atom feels
 * the friction force -m (1/tau_T) (T_i - T_e)/T_i v_i, with T_i = m v_i^2 /
 * (3 k_B) its own kinetic temperature and T_e the electronic temperature
 * (K). The velocity-Verlet steps apply it in two half steps around the
 * force kicks, each the exact solution of the friction term alone
 * (T_i <- T_e + (T_i - T_e) exp(-dt/tau_T), direction kept; an atom at rest
 * stays at rest). tau_T (fs) <= 0 switches it off (the default). Affects the
 * md_step / md_batch_step calls that follow, both schedules and both
 * precisions. Errors: MD_ERR_ARG for a NULL handle, a negative or
 * non-finite T_e or a non-finite tau_T. */
MD_API int md_set_thermostat(md_batch* b, double T_e, double tau_T);

/* Float64 force evaluation with Newton's third law (the paper's CPU scheme,
 * Sec. 4.3) instead of full-list sums: the density and force passes walk
 * only the upper half of each neighbour list (j > i) and add every pair's
 * rho, V and force to both atoms, to the partner by atomic adds (rho and V
 * into the exact fixed-point totals the default path uses, the force in
 * float64). Half the cached bytes and float64 operations of the two sums;
 * the order in which the float64 force atomics land varies, so forces agree
 * with the full-list passes to rounding, not bit for bit, and repeated runs
 * may differ in the last bits (the full-list default is reproducible). Per-atom virials hold
 * each pair once (box pressures are unchanged). on = 0 restores the
 * default. Applies to single-box and tile-schedule steps; the box schedule
 * keeps its own in-shared-memory sums. Errors: MD_ERR_ARG for a NULL
 * handle; MD_ERR_UNSUPPORTED for a mixed-precision handle. */
MD_API int md_set_newton3(md_batch* b, int on);

/* Species of every atom (the type array of Sec. 3.1; Eq. (1)-(3) with
 * type-dependent V, rho and F, Sec. 2), types [n] in caller order (host or device), each
 * in [0, n_types) of the potential; all atoms are species 0 until set.
 * Applies to the current state at once (forces are re-evaluated) and to
 * later state loads. Several species run the tile schedule; their
 * parameter adjoint is not provided (MD_ERR_UNSUPPORTED). Errors:
 * MD_ERR_ARG for a NULL handle or array or a type out of range. */
MD_API int md_set_types(md_batch* b, const int32_t* types, md_stream stream);

/* Instantaneous pressure of Eq. (6) of every box for the current state,
 * P = (N k_B T + W/3)/V in eV/A^3 (1 eV/A^3 = 160.2177 GPa), with T the box's
 * kinetic temperature (3N-3 degrees of freedom) and W = sum_i f_i . r_i the
 * virial of the forces of Eq. (3), written for periodic boxes as the sum
 * over pairs of -(dE_T/dr) r. The forces are re-evaluated with the virial
 * (the same values). p_box: [n_boxes], host or device. Errors: MD_ERR_ARG
 * for a NULL handle or p_box, or before any state was set. */
MD_API int md_pressure(md_batch* b, double* p_box, md_stream stream);

/* Pressure control of Eq. (5) (Berendsen et al.): after every step each
 * box's coordinates and lengths are multiplied by
 * mu = [1 - beta (dt/tau_p)(P0 - P)]^(1/3), P its pressure of Eq. (6) at the
 * end of the step, P0 the target (eV/A^3) and beta the compressibility
 * (A^3/eV) that the printed equation leaves implicit. tau_p (fs) <= 0
 * switches it off (the default). While it is on, md_batch_step uses the
 * tile schedule, a single box runs the batch kernels (its length lives on
 * the device), and a step that would shrink a box below one list radius
 * per cell (the cell grid is fixed at creation) fails with
 * MD_ERR_UNSUPPORTED. md_get_box reads the current lengths. Errors:
 * MD_ERR_ARG for a NULL handle, a non-finite argument, or beta <= 0 with
 * tau_p > 0. */
MD_API int md_set_barostat(md_batch* b, double P0, double tau_p, double beta);

/* Current box lengths [n_boxes][3] (A), as scaled by the coupling of
 * Eq. (5), into a host or device array. */
MD_API int md_get_box(md_batch* b, double* lengths, md_stream stream);

/* Gradient of a scalar loss L with respect to the potential parameters
 * (RGL: A, xi, p, q, r0; spline: all knot values in md_potential's knot
 * order, V then rho then F, each per type pair or type for T > 1), at
 * the batch's current positions, given g_f = dL/dF [n][3] (device, caller
 * order) and g_e = dL/dE_T per box [n_boxes] (device):
 *   grad = sum_i g_f_i . dF_i/dtheta + sum_b g_e_b dE_b/dtheta.
 * The adjoint recomputes rho_i and F'(rho_i) instead of storing per-pair
 * terms. grad [n_param] (device) is overwritten. No counterpart in the
 * paper. MD_ERR_UNSUPPORTED for Sutton-Chen. */
MD_API int md_param_grad(md_batch* b, const double* g_f, const double* g_e, double* grad, md_stream stream);

/* Number of potential parameters of md_param_grad (no counterpart in the
 * paper; 5 for RGL/SC; for a spline the knot
 * count, P (n_phi + n_f) + T n_F with T species and P = T (T + 1) / 2). */
MD_API int md_num_params(const md_batch* b);

/* ---------------------------------------------------------------- profiling */

/* Phases of a step, for md_profile. */
enum md_phase {
    MD_PHASE_KICK_DRIFT = 0, /* first half-kick, drift, displacement check */
    MD_PHASE_REBUILD = 1,    /* binning, sort and list build (early exit when not due) */
    MD_PHASE_PAIRS = 2,      /* float64: pair functions, once per pair, into both lists */
    MD_PHASE_DENSITY = 3,    /* density sums and embedding derivative (mixed: the whole
                                density pass) */
    MD_PHASE_FORCE = 4,      /* force pass and second half-kick (box schedule: all phases) */
    MD_PHASE_OTHER = 5,      /* step bookkeeping, reductions, copies */
    MD_PHASE_GRAD = 6,       /* md_param_grad: the adjoint kernels */
    MD_PHASE_COUNT = 7
};

/* Kernel launches issued by a handle since md_profile_start, and (when
 * timing is on) device time per phase from CUDA events recorded around each
 * phase on the caller's stream. The phases are those of a step of Sec. 3.3
 * (Fig. 4); the paper times the list build and the two force kernels
 * separately in Sec. 4.1-4.2. */
typedef struct md_profile {
    int64_t launches;                 /* kernels launched (graph replays included) */
    double ms[MD_PHASE_COUNT];        /* summed event time per phase, ms */
    int64_t timed[MD_PHASE_COUNT];    /* timed launches per phase */
} md_profile;

/* Resets the counters (phases of Sec. 3.3, as md_profile). timing != 0
 * records events around every phase (and disables CUDA-graph replay while
 * on); timing == 0 only counts launches. */
MD_API int md_profile_start(md_batch* h, int timing);

/* Reads the counters of md_profile_start (phases of Sec. 3.3;
 * synchronizes the device). */
MD_API int md_profile_read(md_batch* h, md_profile* out);

/* Diagnostics (no counterpart in the paper, whose pair functions come from
 * lookup tables, Sec. 3.3): evaluates the library's float64 elementary functions on n
 * values x [n] (device) into out [n] (device): fn 0 = table-driven e^x
 * (arguments |x| < 700), 1 = CUDA exp(x), 2 = 1/sqrt(x) by the library's
 * float32 estimate plus one third-order Newton step (x > 0), 3 = CUDA
 * rsqrt(x), 4 and 5 = 1/sqrt(x) and sqrt(x) as the float64 pair functions
 * take them, a float32 estimate and a third-order Newton step in fixed point
 * on the integer pipe, each rounded once (x positive and normal). Lets a
 * caller bound the error of the hot-path functions.
 * MD_ERR_ARG for an unknown fn or non-device pointers. */
MD_API int md_eval_math(md_batch* h, int fn, const double* x, int64_t n, double* out, md_stream stream);

/* Diagnostics (no counterpart in the paper): the device's fused
 * multiply-add rate, the denominator of the float64 (precision 0) and
 * float32 (precision 1) rooflines of the pair math. Every resident thread
 * (the device full of 256-thread blocks) runs 8 x iters (iters rounded up
 * to a multiple of 16) FMAs x <- x a + b in 4, 8 and then 16 independent
 * chains, one launch each timed with CUDA events on `stream`; the call
 * synchronizes and writes (host) the fastest launch's rate in flop/s (2 per
 * FMA) to *flops, its time in ms to *ms and the multiprocessor count to
 * *n_sm. It allocates a small
 * output array of its own. Errors: MD_ERR_ARG (precision not 0 or 1,
 * iters < 1, a NULL output), MD_ERR_NOMEM, MD_ERR_CUDA. */
MD_API int md_fma_probe(int precision, int64_t iters, double* flops, double* ms, int* n_sm, md_stream stream);

/* ---------------------------------------------------------------- deferred device status */

/* Deferred device status (no counterpart in the paper). With on != 0,
 * md_get_forces, md_batch_thermo, md_batch_set_potential and md_param_grad
 * return once their work is enqueued on `stream` instead of waiting for it
 * to read the device status word: a loop of such calls (a fitting loop)
 * keeps the GPU busy without a host round trip per call. Outputs are valid
 * once the stream reaches the call (host destinations on return, as
 * before). A device-side condition that their kernels raise (a non-finite
 * value, a list overflow) is reported by the next call that waits: md_sync,
 * md_step, md_get_state, md_set_state and every call not listed here, all
 * of which keep waiting. Argument errors are returned at once either way.
 * on = 0 (the default) restores per-call waiting. Errors: MD_ERR_ARG for a
 * NULL handle. */
MD_API int md_set_deferred_status(md_batch* b, int on);

/* Waits for `stream` and reports the device status word: MD_OK, or the
 * condition a deferred call raised (MD_ERR_NONFINITE, MD_ERR_NEIGH_OVERFLOW,
 * MD_ERR_UNSUPPORTED for a pressure-coupled box below one list radius per
 * cell). No counterpart in the paper. Errors: MD_ERR_ARG for a NULL handle,
 * MD_ERR_CUDA. */
MD_API int md_sync(md_batch* b, md_stream stream);

/* ---------------------------------------------------------------- allocation-free variant */

/* Largest atom count md_forces_noalloc accepts (no counterpart in the
 * paper). */
#define MD_NOALLOC_MAX_ATOMS 16384

/* Forces and energies of one small periodic box without allocating any
 * device memory. The paper has no counterpart: this exists for callers that
 * cannot call cudaMalloc, such as plug-ins whose host application owns all
 * device memory through its own pool or memory cap, and latency-bound loops
 * that must not enter the driver's allocator (it can synchronize the device
 * and take unbounded time).
 * The caller passes x [n][3] (device), f [n][3] (device) and, optionally,
 * e_atom [n] and e_total [1] (device; NULL skips them), all memory of the
 * current device (or managed memory); box [3] is a host array; pot must be
 * RGL or Sutton-Chen (MD_ERR_UNSUPPORTED otherwise). With n_atoms == 0, x
 * and f may be NULL and *e_total (when given) is set to 0 on the stream.
 * Results are the forces and energies md_compute_forces gives for the same
 * positions, computed by an all-pairs minimum-image loop, O(n^2) per call,
 * no cells and no list. Positions may lie outside the box (any number of
 * box lengths away); the minimum image is taken by rounding.
 * Working memory is one file-scope device array of 5 * MD_NOALLOC_MAX_ATOMS
 * doubles (640 KiB) that every GPU loading the library holds until the
 * process exits. The first call on a device looks up that array's device
 * address with the device current; make that first call before any stream
 * capture. All calls share the array and each call overwrites the entries
 * it reads before reading them, so nothing needs clearing between calls;
 * calls that overlap on the GPU (for example on two streams) race on it and
 * must be serialized by the caller.
 * Errors: MD_ERR_ARG (n_atoms > MD_NOALLOC_MAX_ATOMS or < 0, a box length not
 * above 2 r_cut, x/f/e_atom/e_total not memory of the current device),
 * MD_ERR_UNSUPPORTED,
 * MD_ERR_CUDA. Asynchronous: outputs are valid once `stream` reaches the
 * call. */
MD_API int md_forces_noalloc(const md_potential* pot, const double* box, int64_t n_atoms, const double* x,
                             double* f, double* e_atom, double* e_total, md_stream stream);

/* ---------------------------------------------------------------- errors */

/* Name of a status code (no counterpart in the paper). */
MD_API const char* md_status_string(int status);
/* Text of the last failure on the handle (or of the last failed create
 * when h is NULL). Valid until the next call on the handle. No counterpart
 * in the paper. */
MD_API const char* md_last_error(const md_batch* h);

#ifdef __cplusplus
}
#endif

#endif /* MD_H */
