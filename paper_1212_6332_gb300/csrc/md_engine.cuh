// Internal declarations of the many-body MD engine (CUDA, sm_103a).
//
// One engine serves a single box and a batch of boxes alike: a single box is
// a batch of one (the paper's multiple-box-in-one-run scheme, Sec. 4.4,
// numbers the cells of box I after those of boxes 0..I-1). Atoms are kept
// sorted by cell, cells of each box in Morton order; boxes are contiguous.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "md.h"
#include "md_math.cuh"

namespace mdk {

// Unit constants (CODATA 2018).
constexpr double kMVV = 103.642696527;  // eV per u (A/fs)^2
constexpr double kBoltz = 8.617333262e-5;  // eV/K

// Device status bits.
constexpr int kStOverflow = 1;
constexpr int kStNonFinite = 2;
constexpr int kStTimeout = 4;
constexpr int kStCellSide = 8;  // a pressure-coupled box shrank below one list radius per cell
constexpr int kSumWords = 4;  // fixed-point density totals: words per atom (rho, V; low and high)

// Potential, passed by value to kernels.
struct Pot {
    int n_types;  // species (splines): V, rho tables per type pair, F per type
    int kind;
    double rc, rc2, rs, inv_w;  // cutoff, taper start, 1/(rc - rs); rs >= rc: hard cut
    double rs2;                 // rs^2: pairs with r^2 <= rs2 have S = 1
    // RGL: V = A2 exp(p - p_r0 r) S, rho = xi2 exp(q2 - q2_r0 r) S
    double A2, xi2, p, p_r0, q2, q2_r0;
    int fold;        // 2A > 0 and xi^2 > 0: exponent constants with the prefactors folded in
    double pA, qX;   // p + ln(2A), 2q + ln(xi^2)
    double xi, r0;  // RGL xi and r0 (parameter derivatives)
    // SC: V = eps (a/r)^n S, rho = (a/r)^m S; F = -F_scale sqrt(rho)
    double eps, a, n, m;
    int sc96;        // SC exponents n = 9, m = 6: (a/r)^9 and (a/r)^6 from one chain of products
    double F_scale;
    // spline: per-interval cubic coefficients (c0 + c1 u + c2 u^2 + c3 u^3,
    // u = t - t_k) for V, rho, F; n knots -> n - 1 intervals
    const double4_32a* sp[3];
    int sn[3];
    double st0[3], sh[3], sinvh[3];
    // the same coefficients rounded to float32 (mixed-precision path: no
    // float64 loads or conversions per evaluation)
    const float4* spf[3];
    float st0f[3], shf[3], sinvhf[3];
    // float64 pair path when V and rho share one grid (n_phi == n_f): per
    // type pair n + 1 records of 16 doubles (128 bytes), record 0 the linear
    // continuation below r_lo, records 1..n-1 the intervals, record n the
    // linear continuation above r_hi; each record holds
    //   (t_k, v0, v1, v2 | v3, 2 v2, 3 v3, f0 | f1, f2, f3, 2 f2 | 3 f3, 0, 0, 0)
    // so that V, V', rho, rho' at u = r - t_k take 10 float64 instructions
    // and the interval is found from a float32 copy of r
    const double4_32a* sq;  // null: V and rho on different grids
    int sq_n;               // knots per table (records per table: sq_n + 1)
    float sq_invhf, sq_c0f; // 1/h and -r_lo/h in float32
    // table-driven exponential (float64 path)
    ExpConst ek;
    const double* exp_T;  // [kExpTable] 2^(j/kExpTable)
    // RGL float64 pair path: both exponentials from one table over r,
    // r = k h + d (h = 1/kRxPerA, k the nearest integer, |d| <= h/2):
    //   e_1(r) = E1_k (1 + d R_1(d)),  E1_k = 2A exp(p - p_r0 k h),
    // R_1 the degree-3 Taylor remainder of exp(-p_r0 d) (truncation below
    // 4e-16 relative); the same for rho with (xi^2, 2q, 2q/r0). Entries
    // cover k in [rx_k0, rx_k0 + rx_n); other r take exp_tab.
    const double2* rx;  // [rx_n] (E1_k, E2_k); null: no table
    int rx_k0, rx_n;
    double rx_c1[4], rx_c2[4];  // R_1, R_2 coefficients: -b, b^2/2, -b^3/6, b^4/24
    float rx_f1[2], rx_f2[2];   // float32 copies of the d^3 and d^4 coefficients
    // float copies for the mixed-precision path
    float f_rc2, f_rs, f_inv_w, f_A2, f_xi2, f_p, f_p_r0, f_q2, f_q2_r0, f_eps, f_a, f_n, f_m;
    // mixed RGL in base 2: exp(p - p_r0 r) = 2^(f_g1[0] + f_g1[1] r) and the
    // same for (2q, 2q/r0) in f_g2; taper variable x = sat(r inv_w + f_x0)
    // and dS/dx inv_w = x^2 (f_dS[0] + x (f_dS[1] + x f_dS[2]))
    float f_g1[2], f_g2[2], f_x0, f_dS[3];
};

// Geometry of the boxes, passed by value to kernels.
struct Geo {
    int B;                    // number of boxes
    const double* L;          // [B*3] box lengths
    const double* cell_len;   // [B*3] cell sides
    const float* cell_len_f;  // [B*3] cell sides as float
    const int* nc;            // [B*3] cells per axis
    const int* cell_off;      // [B+1] first global cell of each box
    const int64_t* atom_off;  // [B+1] first atom of each box
    const int* atom_box;      // [N] box of each atom slot
    const int* cell_box;      // [n_cells] box of each global cell
    const int* cell_rank;     // [n_cells] (box, row-major cell) -> global Morton-ordered cell
    const int* cell_xyz;      // [n_cells] global cell -> packed (cx | cy << 10 | cz << 20)
    const double4_32a* cell_org;  // [n_cells] cell origin (x, y, z) and, in w's bits, the packed coordinates
    // single-box fast path
    double L0[3];
};

// Device-resident control words.
struct Ctl {
    int status;                      // kSt* bits
    int overflow_count;              // largest neighbour count seen at overflow
    unsigned long long disp2_last;   // largest squared displacement of the last step (double bits)
    long long step;                  // completed steps since set_state
    long long n_rebuild;             // list builds since set_state
    int max_count;                   // largest neighbour count of the current list
    int n_due;                       // cells queued for a partial list build
    unsigned long long n_gate_skip;  // graph-replayed steps whose rebuild body the gate skipped (never reset)
    int pos_changed;                 // a state load that kept the lists met a position unlike the current one
};

// Electron-phonon friction of Eq. (4) over one half step (off unless on):
// each atom's kinetic temperature T_i = m_3kb v^2 relaxes towards T_e by
// the exact factor of the friction term alone, T_i <- T_e + (T_i - T_e)
// decay with decay = exp(-dt/tau_T), along the fixed direction of v.
struct Bath {
    double T_e;    // electronic temperature (K)
    double decay;  // exp(-2 (dt/2) / tau_T)
    double m_3kb;  // m / (3 k_B) in K per (A/fs)^2
    int on;
};

// Berendsen pressure coupling of Eq. (5): after each step every box's
// coordinates and lengths are scaled by mu = [1 - beta (dt/tau_p)(P0 - P)]^(1/3)
// with P the box's instantaneous pressure of Eq. (6).
struct Baro {
    double P0;        // target pressure (eV/A^3)
    double k;         // beta dt / tau_p (A^3/eV)
    int on;
};

// Float32 cell geometry of a box (mixed-precision separations).
struct CellSep {
    float lx, ly, lz;     // cell sides
    int nx, ny, nz;       // cells per axis
    float Lx, Ly, Lz;     // box lengths
};

// Shared-memory size class of the block-per-box schedule.
struct BoxClass {
    int first, count, threads;
    size_t smem;
};

struct Engine {
    // configuration
    md_config cfg{};
    md_potential pot_host{};
    std::vector<double> knots_host;
    Pot pot{};
    int B = 0;
    int64_t N = 0, N_pad = 0;
    int n_cells = 0;
    int max_nb = 0;
    bool wide = false;  // every box has at least 3 cells per axis
    int n_sm = 1;       // multiprocessors of the handle's device
    double rl = 0.0;  // list radius r_cut + skin
    std::vector<int64_t> atom_off_h;
    std::vector<double> L_h;
    std::vector<int> nc_h, cell_off_h;
    std::string err;

    // geometry tables (device)
    double* L = nullptr;
    double* cell_len = nullptr;
    float* cell_len_f = nullptr;
    int* nc = nullptr;
    int* cell_off = nullptr;
    int64_t* atom_off = nullptr;
    int* atom_box = nullptr;
    int* cell_box = nullptr;
    int* cell_rank = nullptr;
    int* cell_xyz = nullptr;
    double4_32a* cell_org = nullptr;
    double4_32a* spline_coef = nullptr;  // 3 splines back to back
    float4* spline_coef_f = nullptr;     // the same, float32
    double4_32a* spline_pair_rec = nullptr;  // [P][n_phi + 1][4] float64 pair records (n_phi == n_f only)
    double2* rx_tab = nullptr;               // RGL: [rx_n] exponential table over r (Pot.rx)
    std::vector<double2> rx_host;            // its host copy (kept alive for the upload)
    double* spline_work = nullptr;   // [3 * total knots] setup scratch
    double* knots_dev = nullptr;
    // reduction chunks: (box, [lo, hi)) pieces of at most 4096 atoms
    int n_chunks = 0;
    int64_t* chunk_lo = nullptr;
    int64_t* chunk_hi = nullptr;
    int* box_chunk_off = nullptr;  // [B+1]

    // atoms, sorted order (device)
    double4_32a* x = nullptr;    // positions (w unused)
    double4_32a* x_alt = nullptr;
    double4_32a* xb = nullptr;   // positions at the last list build
    double* v = nullptr;     // [3][N_pad] SoA
    double* v_alt = nullptr;
    double* f = nullptr;     // [3][N_pad] SoA
    double* rho = nullptr;
    double* Fp = nullptr;
    float4* xf = nullptr;    // mixed: cell-local offset with float32 F'(rho) in w
    double* e_atom = nullptr;
    float4* xo = nullptr;    // mixed: cell-local offsets, w = packed cell coords
    longlong4_32a* xq = nullptr;  // float64 pair pass: fixed-point positions (x 2^kq) and species
    long long* sum_q = nullptr;   // float64 density sums: fixed-point totals of rho_i and sum_j V_ij, 4 words x N_pad
    int* perm = nullptr;     // sorted slot -> caller index
    int* perm_alt = nullptr;
    int* iperm = nullptr;    // caller index -> sorted slot
    int* cell_of = nullptr;  // [N] global cell of each slot (binning, old order)
    int* cell_t = nullptr;      // [N] cell of each sorted slot at the last build
    int* cell_t_alt = nullptr;
    int* src = nullptr;      // [N] new slot -> old slot
    int* cell_count = nullptr;  // [n_cells] zero at rest
    int* cell_start = nullptr;  // [n_cells + 1]
    int* scan_tmp = nullptr;
    int* nn = nullptr;          // [N_pad]
    int* nl = nullptr;          // [max_nb][N_pad] column-major
    // float64 path: [max_nb][N_pad] pair cache, per list entry (V'/r, rho'/r,
    // rho(r), V(r)) in one 32-byte sector, so the scattered mirror writes of
    // the pair pass are whole sectors (no read-modify-write fills)
    double4_32a* pc = nullptr;
    int* rev = nullptr;         // float64 path: [max_nb][N_pad] partner position of upper entries
    int* nl_lo = nullptr;       // float64 path: [N_pad][max_nb] row-major lower parts (reverse-index search)
    int* n_up = nullptr;        // float64 path: [N_pad] upper entries of each list (lists are [upper | lower])
    double* exp_T = nullptr;    // exponential table
    // parameter adjoint work arrays (allocated on the first gradient call)
    double* grad_g = nullptr;        // [3][N_pad] dL/dF in sorted order
    double* grad_u = nullptr;        // [N_pad] adjoint scalar u_i
    double* grad_Fpp = nullptr;      // [N_pad] F''(rho_i)
    double* grad_partial = nullptr;  // [grad_blocks][n_coef or 5]
    double* grad_coef = nullptr;     // spline coefficient gradients
    int grad_blocks = 0;
    ExpConst exp_const{};
    double* stage = nullptr;    // [3N] staging for host copies / caller-order outputs
    double* red = nullptr;      // reduction scratch [2 * n_chunks]
    double* thermo_dev = nullptr;  // [B][4] + [4] totals
    double* hist = nullptr;        // per-step thermo ring
    int hist_cap = 0;
    Ctl* ctl = nullptr;
    Ctl* ctl_host = nullptr;       // pinned mirror
    unsigned long long* disp_box = nullptr;  // [B] largest squared displacement since the box's last build
    int* due_cells = nullptr;                // [n_cells] cells of the boxes a partial build renews

    bool have_state = false;
    bool lists_ok = false;  // lists, cells and build positions agree (a state load may keep them)
    bool forces_ok = false; // f, rho, F', e_atom are those of the current positions (not after a box scaling)
    Bath bath{};            // friction of Eq. (4) applied in the kicks (md_set_thermostat)
    bool newton3 = false;   // float64 half-list sums with Newton's third law (md_set_newton3)
    // captured steps skip their rebuild kernels through a graph conditional
    // node when no box is due (cond_off: the capture fell back to plain
    // launches); the launch count subtracts the skipped bodies
    bool cond_off = false;
    long long graph_body_kernels = 0;
    unsigned long long gate_skip_seen = 0;
    Baro baro{};            // pressure coupling of Eq. (5) after each step (md_set_barostat)
    int* types = nullptr;   // [N] species of each atom, caller order (md_set_types; 0 by default)
    double* w_atom = nullptr;   // [N_pad] per-atom virial -1/2 sum_j s_ij r_ij^2 (pressure users only)
    double* red_w = nullptr;    // [n_chunks] chunk sums of w_atom
    double* press_box = nullptr;  // [B] pressure of each box (eV/A^3)
    double* mu_box = nullptr;     // [B] scaling factor of the last coupled step
    // CUDA graph of one step (and of a chunk of steps)
    cudaGraphExec_t graph_step = nullptr;
    cudaGraphExec_t graph_chunk = nullptr;
    cudaGraphExec_t graph_last = nullptr;  // one step that forms the pair-energy sums (the last of a run)
    int graph_chunk_len = 0;
    bool graph_hist = false;
    int sched_choice = 0;  // autotuner result for batches (0 = unknown)
    double sched_ms[2] = {0.0, 0.0};  // autotuner timings per step: tile, box
    // block-per-box schedule
    int* box_order = nullptr;
    int* box_done = nullptr;
    int* box_state = nullptr;
    std::vector<BoxClass> box_classes;
    long long graph_chunk_kernels = 0, graph_step_kernels = 0, graph_last_kernels = 0;
    // whether the next float64 force evaluation adds V(r) into the
    // fixed-point pair-energy totals: off for the steps of a run before its
    // last when no step records its energy (dynamics needs rho_i, F and F'
    // only; the energies are read after the last step)
    bool pair_energy = true;
    // md_set_deferred_status: the calls that only wait to read the device
    // status word return without waiting
    bool deferred_status = false;

    // profiling: launch counter and phase events
    long long launches = 0;
    bool prof_timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_phase;
    size_t ev_used = 0;  // pairs in use
};

// Records a start event for `phase` when timing is on; returns the pair index.
inline int prof_begin(Engine& e, int phase, cudaStream_t s) {
    if (!e.prof_timing) return -1;
    if (2 * (e.ev_used + 1) > e.ev_pool.size()) {
        for (int k = 0; k < 2; ++k) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) return -1;
            e.ev_pool.push_back(ev);
        }
    }
    int idx = (int)e.ev_used++;
    if (e.ev_phase.size() <= (size_t)idx) e.ev_phase.resize(idx + 1);
    e.ev_phase[idx] = phase;
    cudaEventRecord(e.ev_pool[2 * idx], s);
    return idx;
}

inline void prof_end(Engine& e, int idx, cudaStream_t s) {
    if (idx >= 0) cudaEventRecord(e.ev_pool[2 * idx + 1], s);
}

// Scope guard: events around the launches of one phase.
struct PhaseScope {
    Engine& e;
    cudaStream_t s;
    int idx;
    PhaseScope(Engine& e_, int phase, cudaStream_t s_) : e(e_), s(s_), idx(prof_begin(e_, phase, s_)) {}
    ~PhaseScope() { prof_end(e, idx, s); }
};

Geo make_geo(const Engine& e);
// float32 cell geometry of a single-box handle (batches read it per box)
CellSep single_cell_sep(const Engine& e);

// ---- kernels' host launchers (all enqueue on `s`) ----
// binning + sort + permute + list build; mode 1 = always, 0 = only when the
// device displacement word exceeds (skin/2)^2
void launch_rebuild(Engine& e, int mode, cudaStream_t s);
void launch_rebuild_gate(Engine& e, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_build_list(Engine& e, int mode, cudaStream_t s);
// density and force passes (fp64 or mixed); kick != 0 fuses v += dt/2 F/m
void launch_forces(Engine& e, int kick, cudaStream_t s, bool virial = false);
// A single box runs the specialised single-box kernels unless its length
// changes on the device (pressure coupling), where the batch kernels read it.
inline bool single_fast(const Engine& e) { return e.B == 1 && !e.baro.on; }
// Pressure of every box from the per-atom virial of the last force pass
// (and, when coupled, the scaling of Eq. (5)); needs launch_thermo first.
void launch_pressure(Engine& e, bool couple, cudaStream_t s);
void launch_kick_drift(Engine& e, cudaStream_t s);
void launch_end_step(Engine& e, int record_hist, cudaStream_t s);
void launch_thermo(Engine& e, cudaStream_t s);
void launch_thermo_hist(Engine& e, cudaStream_t s);
void launch_reset_ctl(Engine& e, cudaStream_t s);
void launch_prepare_mixed(Engine& e, cudaStream_t s);
void launch_spline_setup(Engine& e, cudaStream_t s);
// caller-order <-> sorted-order copies
void launch_load_positions(Engine& e, const double* src_caller, cudaStream_t s);
void launch_load_positions_keep(Engine& e, const double* src_caller, cudaStream_t s);
void launch_after_load(Engine& e, cudaStream_t s);
void launch_apply_types(Engine& e, cudaStream_t s);
void launch_load_velocities(Engine& e, const double* src_caller, cudaStream_t s);
void launch_store_vec(Engine& e, const double* soa_or_null, const double4_32a* x4_or_null, double* dst_caller,
                      cudaStream_t s);
void launch_store_scalar(Engine& e, const double* src_sorted, double* dst_caller, cudaStream_t s);
void launch_get_neighbors(Engine& e, int32_t* nn_out, int32_t* nl_out, int32_t ld, cudaStream_t s);
void launch_box_energy(Engine& e, double* e_box_dev, cudaStream_t s);
void launch_reset_perm(Engine& e, cudaStream_t s);
void launch_eval_math(Engine& e, int fn, const double* x, int64_t n, double* out, cudaStream_t s);
// batched block-per-box schedule
int launch_box_steps(Engine& e, int n_steps, bool first, cudaStream_t s);
void launch_advance_steps(Engine& e, long long n, cudaStream_t s);
bool box_schedule_fits(const Engine& e);
// parameter adjoint
int launch_param_grad(Engine& e, const double* g_f, const double* g_e, double* grad, cudaStream_t s);

}  // namespace mdk
