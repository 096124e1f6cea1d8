// Host side of the C ABI declared in md.h: argument checks, device buffers,
// Morton-ordered cell tables, state transfer in caller order, the step loop
// with a device-side rebuild decision, neighbour-overflow recovery and CUDA
// graph replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "md_engine.cuh"

using namespace mdk;

struct md_batch {
    Engine e;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t body_stream = nullptr;  // captures the conditional rebuild bodies
};

static thread_local std::string g_err;

namespace mdk {

Geo make_geo(const Engine& e) {
    Geo g{};
    g.B = e.B;
    g.L = e.L;
    g.cell_len = e.cell_len;
    g.cell_len_f = e.cell_len_f;
    g.nc = e.nc;
    g.cell_off = e.cell_off;
    g.atom_off = e.atom_off;
    g.atom_box = e.atom_box;
    g.cell_box = e.cell_box;
    g.cell_rank = e.cell_rank;
    g.cell_xyz = e.cell_xyz;
    g.cell_org = e.cell_org;
    for (int a = 0; a < 3; ++a) g.L0[a] = e.L_h.size() >= 3 ? e.L_h[a] : 0.0;
    return g;
}

}  // namespace mdk

namespace {

int fail(Engine* e, int code, const std::string& msg) {
    if (e) {
        e->err = msg;
        e->forces_ok = false;
    } else {
        g_err = msg;
    }
    return code;
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t ck_ = (call);                                                              \
        if (ck_ != cudaSuccess) return fail(E, MD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(ck_)); \
    } while (0)

bool finite(double v) { return std::isfinite(v); }

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
int dalloc(Engine* E, T** p, size_t count) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(E, MD_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    return MD_OK;
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

int check_potential(const md_potential* p, std::string& why) {
    if (!p) return why = "potential is NULL", MD_ERR_ARG;
    if (p->kind == MD_POT_RGL || p->kind == MD_POT_SC) {
        for (int k = 0; k < 5; ++k)
            if (!finite(p->p[k])) return why = "non-finite potential parameter", MD_ERR_ARG;
        if (!(p->r_cut > 0.0) || !finite(p->r_cut) || !finite(p->r_taper))
            return why = "r_cut must be positive and finite", MD_ERR_ARG;
        if (p->kind == MD_POT_RGL && !(p->p[4] > 0.0)) return why = "RGL r0 must be positive", MD_ERR_ARG;
        if (p->kind == MD_POT_SC && !(p->p[2] > 0.0)) return why = "Sutton-Chen a must be positive", MD_ERR_ARG;
        if (p->kind == MD_POT_RGL) {
            // exponent arguments p - p r/r0 and 2q - 2q r/r0 over 0 <= r < r_cut
            double pp = p->p[2], q2 = 2.0 * p->p[3], r0 = p->p[4], rc = p->r_cut;
            double lo = std::min({pp, pp - pp / r0 * rc, q2, q2 - q2 / r0 * rc});
            double hi = std::max({pp, pp - pp / r0 * rc, q2, q2 - q2 / r0 * rc});
            if (!(lo > -700.0 && hi < 700.0)) return why = "RGL exponents out of range (|arg| >= 700)", MD_ERR_ARG;
        }
        return MD_OK;
    }
    if (p->n_types < 0 || p->n_types > 4) return why = "n_types must be 0..4", MD_ERR_ARG;
    if (p->n_types > 1 && p->kind != MD_POT_SPLINE) return why = "several species need spline tables", MD_ERR_ARG;
    if (p->kind == MD_POT_SPLINE) {
        if (!p->knots) return why = "spline knots are NULL", MD_ERR_ARG;
        if (p->n_phi < 4 || p->n_f < 4 || p->n_F < 4) return why = "each spline needs >= 4 knots", MD_ERR_ARG;
        if (!(p->r_hi > p->r_lo) || !(p->r_lo > 0.0) || !finite(p->r_hi))
            return why = "spline needs 0 < r_lo < r_hi", MD_ERR_ARG;
        if (!(p->rho_hi > p->rho_lo) || !finite(p->rho_lo) || !finite(p->rho_hi))
            return why = "spline needs rho_lo < rho_hi", MD_ERR_ARG;
        return MD_OK;
    }
    return why = "unknown potential kind " + std::to_string(p->kind), MD_ERR_ARG;
}

double pot_cutoff(const md_potential* p) { return p->kind == MD_POT_SPLINE ? p->r_hi : p->r_cut; }

// species, type-pair tables and knot values of a potential
static int pot_types(const md_potential& p) { return p.kind == MD_POT_SPLINE && p.n_types > 1 ? p.n_types : 1; }
static int pot_pairs(const md_potential& p) { return pot_types(p) * (pot_types(p) + 1) / 2; }
static size_t knot_count(const md_potential& p) {
    return (size_t)pot_pairs(p) * (p.n_phi + p.n_f) + (size_t)pot_types(p) * p.n_F;
}

void fill_pot(Engine& e) {
    const md_potential& p = e.pot_host;
    Pot P{};
    P.kind = p.kind;
    P.n_types = pot_types(p);
    if (p.kind == MD_POT_SPLINE) {
        P.rc = p.r_hi;
        P.rs = p.r_hi;
        P.inv_w = 0.0;
        int ns[3] = {p.n_phi, p.n_f, p.n_F};
        int ntab[3] = {pot_pairs(p), pot_pairs(p), pot_types(p)};  // tables of V, rho, F
        double lo[3] = {p.r_lo, p.r_lo, p.rho_lo}, hi[3] = {p.r_hi, p.r_hi, p.rho_hi};
        size_t off = 0;
        for (int w = 0; w < 3; ++w) {
            P.sp[w] = e.spline_coef + off;
            P.spf[w] = e.spline_coef_f + off;
            P.sn[w] = ns[w];
            P.st0[w] = lo[w];
            P.sh[w] = (hi[w] - lo[w]) / (ns[w] - 1);
            P.sinvh[w] = 1.0 / P.sh[w];
            P.st0f[w] = (float)P.st0[w];
            P.shf[w] = (float)P.sh[w];
            P.sinvhf[w] = (float)P.sinvh[w];
            off += (size_t)ntab[w] * ns[w];
        }
        P.sq = e.spline_pair_rec;
        P.sq_n = p.n_phi;
        P.sq_invhf = (float)P.sinvh[0];
        P.sq_c0f = (float)(-p.r_lo * P.sinvh[0]);
    } else {
        P.rc = p.r_cut;
        if (p.r_taper < p.r_cut) {
            P.rs = p.r_taper;
            P.inv_w = 1.0 / (p.r_cut - p.r_taper);
        } else {
            P.rs = p.r_cut;
            P.inv_w = 0.0;
        }
    }
    P.rc2 = P.rc * P.rc;
    P.rs2 = P.rs * P.rs;
    P.F_scale = 1.0;
    if (p.kind == MD_POT_RGL) {
        double A = p.p[0], xi = p.p[1], pp = p.p[2], q = p.p[3], r0 = p.p[4];
        P.A2 = 2.0 * A;
        P.xi2 = xi * xi;
        P.p = pp;
        P.p_r0 = pp / r0;
        P.q2 = 2.0 * q;
        P.q2_r0 = 2.0 * q / r0;
        P.xi = xi;
        P.r0 = r0;
        P.fold = P.A2 > 0.0 && P.xi2 > 0.0;
        P.pA = P.fold ? pp + std::log(P.A2) : 0.0;
        P.qX = P.fold ? P.q2 + std::log(P.xi2) : 0.0;
    } else if (p.kind == MD_POT_SC) {
        P.eps = p.p[0];
        P.a = p.p[2];
        P.n = p.p[3];
        P.m = p.p[4];
        P.sc96 = P.n == 9.0 && P.m == 6.0;
        P.F_scale = p.p[1] * p.p[0];
    }
    P.ek = e.exp_const;
    P.exp_T = e.exp_T;
    if (p.kind == MD_POT_RGL && e.rx_tab) {
        // r table from 0.3 r_cut (closer pairs take exp_tab) to past r_cut
        P.rx = e.rx_tab;
        P.rx_k0 = (int)std::floor(0.3 * P.rc * kRxPerA);
        P.rx_n = (int)std::ceil(P.rc * kRxPerA) + 2 - P.rx_k0;
        const double b[2] = {P.p_r0, P.q2_r0};
        double* c[2] = {P.rx_c1, P.rx_c2};
        for (int f = 0; f < 2; ++f) {
            c[f][0] = -b[f];
            c[f][1] = b[f] * b[f] / 2.0;
            c[f][2] = -b[f] * b[f] * b[f] / 6.0;
            c[f][3] = b[f] * b[f] * b[f] * b[f] / 24.0;
        }
        P.rx_f1[0] = (float)P.rx_c1[2];
        P.rx_f1[1] = (float)P.rx_c1[3];
        P.rx_f2[0] = (float)P.rx_c2[2];
        P.rx_f2[1] = (float)P.rx_c2[3];
    }
    P.f_rc2 = (float)P.rc2;
    P.f_rs = (float)P.rs;
    P.f_inv_w = (float)P.inv_w;
    P.f_A2 = (float)P.A2;
    P.f_xi2 = (float)P.xi2;
    P.f_p = (float)P.p;
    P.f_p_r0 = (float)P.p_r0;
    P.f_q2 = (float)P.q2;
    P.f_q2_r0 = (float)P.q2_r0;
    P.f_eps = (float)P.eps;
    P.f_a = (float)P.a;
    P.f_n = (float)P.n;
    P.f_m = (float)P.m;
    const double log2e = 1.4426950408889634;
    P.f_g1[0] = (float)(P.p * log2e);
    P.f_g1[1] = (float)(-P.p_r0 * log2e);
    P.f_g2[0] = (float)(P.q2 * log2e);
    P.f_g2[1] = (float)(-P.q2_r0 * log2e);
    P.f_x0 = (float)(-P.rs * P.inv_w);
    P.f_dS[0] = (float)(-30.0 * P.inv_w);
    P.f_dS[1] = (float)(60.0 * P.inv_w);
    P.f_dS[2] = (float)(-30.0 * P.inv_w);
    e.pot = P;
}

uint64_t spread3(uint64_t v) {
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
}

void destroy_graphs(Engine& e) {
    if (e.graph_step) cudaGraphExecDestroy(e.graph_step);
    if (e.graph_chunk) cudaGraphExecDestroy(e.graph_chunk);
    if (e.graph_last) cudaGraphExecDestroy(e.graph_last);
    e.graph_step = e.graph_chunk = e.graph_last = nullptr;
}

void free_engine(Engine& e) {
    destroy_graphs(e);
    dfree(e.L); dfree(e.cell_len); dfree(e.cell_len_f); dfree(e.nc); dfree(e.cell_off); dfree(e.atom_off);
    dfree(e.atom_box); dfree(e.cell_box); dfree(e.cell_rank); dfree(e.cell_xyz); dfree(e.cell_org); dfree(e.spline_coef); dfree(e.spline_coef_f);
    dfree(e.spline_work); dfree(e.spline_pair_rec); dfree(e.rx_tab); dfree(e.knots_dev); dfree(e.chunk_lo); dfree(e.chunk_hi); dfree(e.box_chunk_off);
    dfree(e.x); dfree(e.x_alt); dfree(e.xb); dfree(e.v); dfree(e.v_alt); dfree(e.f); dfree(e.rho); dfree(e.Fp);
    dfree(e.xf); dfree(e.e_atom); dfree(e.xo); dfree(e.xq); dfree(e.sum_q); dfree(e.perm); dfree(e.perm_alt); dfree(e.iperm);
    dfree(e.cell_of); dfree(e.cell_t); dfree(e.cell_t_alt); dfree(e.src); dfree(e.cell_count);
    dfree(e.cell_start); dfree(e.scan_tmp); dfree(e.nn); dfree(e.nl); dfree(e.pc); dfree(e.rev); dfree(e.nl_lo); dfree(e.n_up); dfree(e.exp_T);
    dfree(e.box_order); dfree(e.box_done); dfree(e.box_state);
    dfree(e.grad_g); dfree(e.grad_u); dfree(e.grad_Fpp); dfree(e.grad_partial); dfree(e.grad_coef); dfree(e.stage); dfree(e.red);
    dfree(e.thermo_dev); dfree(e.hist); dfree(e.ctl); dfree(e.disp_box); dfree(e.types); dfree(e.due_cells); dfree(e.w_atom); dfree(e.red_w); dfree(e.press_box); dfree(e.mu_box);
    for (cudaEvent_t ev : e.ev_pool) cudaEventDestroy(ev);
    e.ev_pool.clear();
    if (e.ctl_host) cudaFreeHost(e.ctl_host);
    e.ctl_host = nullptr;
}

int upload_potential(md_batch* h, cudaStream_t s) {
    Engine* E = &h->e;
    Engine& e = *E;
    fill_pot(e);
    if (e.pot.rx) {
        // E_k = 2A exp(p - p_r0 r_k), xi^2 exp(2q - (2q/r0) r_k) at r_k = k h;
        // the exponent with one rounding (fma), exp from the C library
        const Pot& P = e.pot;
        e.rx_host.resize(P.rx_n);
        for (int k = 0; k < P.rx_n; ++k) {
            const double rk = (P.rx_k0 + k) / kRxPerA;
            e.rx_host[k] = make_double2(P.A2 * std::exp(std::fma(-P.p_r0, rk, P.p)),
                                        P.xi2 * std::exp(std::fma(-P.q2_r0, rk, P.q2)));
        }
        CK(cudaMemcpyAsync(e.rx_tab, e.rx_host.data(), P.rx_n * sizeof(double2), cudaMemcpyHostToDevice, s));
    }
    if (e.pot_host.kind == MD_POT_SPLINE) {
        size_t nk = knot_count(e.pot_host);
        CK(cudaMemcpyAsync(e.knots_dev, e.knots_host.data(), nk * sizeof(double), cudaMemcpyHostToDevice, s));
        launch_spline_setup(e, s);
        CK(cudaGetLastError());
    }
    return MD_OK;
}

int create_impl(const md_config* cfg, const md_potential* pot, int B, const int64_t* atom_off, const double* box,
                md_batch** out) {
    Engine* E = nullptr;
    if (!out) return fail(nullptr, MD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, MD_ERR_ARG, "config is NULL");
    std::string why;
    if (check_potential(pot, why) != MD_OK) return fail(nullptr, MD_ERR_ARG, why);
    if (!(cfg->skin >= 0.0) || !finite(cfg->skin)) return fail(nullptr, MD_ERR_ARG, "skin must be >= 0");
    if (!(cfg->dt >= 0.0) || !finite(cfg->dt)) return fail(nullptr, MD_ERR_ARG, "dt must be >= 0");
    if (!(cfg->mass > 0.0) || !finite(cfg->mass)) return fail(nullptr, MD_ERR_ARG, "mass must be > 0");
    if (cfg->precision != MD_FP64 && cfg->precision != MD_MIXED)
        return fail(nullptr, MD_ERR_ARG, "unknown precision");
    if (cfg->max_neighbors < 0) return fail(nullptr, MD_ERR_ARG, "max_neighbors must be >= 0");
    if (B < 1) return fail(nullptr, MD_ERR_ARG, "need at least one box");
    if (!atom_off || atom_off[0] != 0) return fail(nullptr, MD_ERR_ARG, "atom_offsets[0] must be 0");
    for (int b = 0; b < B; ++b)
        if (atom_off[b + 1] < atom_off[b]) return fail(nullptr, MD_ERR_ARG, "atom_offsets must not decrease");
    if (atom_off[B] >= ((int64_t)1 << 26)) return fail(nullptr, MD_ERR_ARG, "at most 2^26 - 1 atoms per handle");
    double rl = pot_cutoff(pot) + cfg->skin;
    for (int b = 0; b < 3 * B; ++b) {
        if (!(box[b] > 0.0) || !finite(box[b])) return fail(nullptr, MD_ERR_ARG, "box lengths must be > 0");
        if (!(rl < 0.5 * box[b]))
            return fail(nullptr, MD_ERR_ARG,
                        "r_cut + skin must be below half of every box length (minimum image)");
    }

    md_batch* h = new (std::nothrow) md_batch();
    if (!h) return fail(nullptr, MD_ERR_NOMEM, "host allocation failed");
    E = &h->e;
    Engine& e = *E;
    e.cfg = *cfg;
    e.pot_host = *pot;
    if (pot->kind == MD_POT_SPLINE) {
        size_t nk = knot_count(*pot);
        e.knots_host.assign(pot->knots, pot->knots + nk);
        e.pot_host.knots = nullptr;
    }
    e.B = B;
    e.N = atom_off[B];
    e.N_pad = std::max<int64_t>(32, (e.N + 31) / 32 * 32);
    e.rl = rl;
    e.atom_off_h.assign(atom_off, atom_off + B + 1);
    e.L_h.assign(box, box + 3 * B);

    // cells: largest count per axis with side >= rl, Morton order inside a box
    e.nc_h.resize(3 * B);
    e.cell_off_h.assign(B + 1, 0);
    std::vector<double> cl(3 * B);
    std::vector<float> clf(3 * B);
    int64_t tot = 0;
    for (int b = 0; b < B; ++b) {
        int64_t nb = 1;
        for (int a = 0; a < 3; ++a) {
            int n = (int)std::floor(box[3 * b + a] / (rl * (1.0 + 1e-12)));
            n = std::max(1, std::min(n, 1023));
            e.nc_h[3 * b + a] = n;
            cl[3 * b + a] = box[3 * b + a] / n;
            clf[3 * b + a] = (float)cl[3 * b + a];
            nb *= n;
        }
        tot += nb;
        if (tot > (int64_t)INT32_MAX / 2) {
            delete h;
            return fail(nullptr, MD_ERR_ARG, "too many cells");
        }
        e.cell_off_h[b + 1] = (int)tot;
    }
    e.n_cells = (int)tot;
    e.wide = *std::min_element(e.nc_h.begin(), e.nc_h.end()) >= 3;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&e.n_sm, cudaDevAttrMultiProcessorCount, dev);
        e.n_sm = std::max(e.n_sm, 1);
    }
    std::vector<int> rank(tot), xyz(tot), cbox(tot);
    for (int b = 0; b < B; ++b) {
        int nx = e.nc_h[3 * b], ny = e.nc_h[3 * b + 1], nz = e.nc_h[3 * b + 2];
        int off = e.cell_off_h[b];
        int n = nx * ny * nz;
        std::vector<std::pair<uint64_t, int>> key(n);
        for (int cx = 0; cx < nx; ++cx)
            for (int cy = 0; cy < ny; ++cy)
                for (int cz = 0; cz < nz; ++cz) {
                    int lin = (cx * ny + cy) * nz + cz;
                    key[lin] = {spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2), lin};
                }
        std::sort(key.begin(), key.end());
        for (int r = 0; r < n; ++r) {
            int lin = key[r].second;
            int cz = lin % nz, cy = (lin / nz) % ny, cx = lin / (ny * nz);
            rank[off + lin] = off + r;
            xyz[off + r] = cx | (cy << 10) | (cz << 20);
            cbox[off + r] = b;
        }
    }
    std::vector<int> abox(e.N);
    std::vector<int64_t> clo, chi;
    std::vector<int> bco(B + 1, 0);
    int64_t max_box = 0;
    double max_dens = 0.0;
    const int64_t CH = 4096;
    for (int b = 0; b < B; ++b) {
        int64_t a0 = atom_off[b], a1 = atom_off[b + 1];
        for (int64_t i = a0; i < a1; ++i) abox[i] = b;
        for (int64_t lo = a0; lo < a1; lo += CH) {
            clo.push_back(lo);
            chi.push_back(std::min(a1, lo + CH));
        }
        bco[b + 1] = (int)clo.size();
        max_box = std::max(max_box, a1 - a0);
        double vol = box[3 * b] * box[3 * b + 1] * box[3 * b + 2];
        max_dens = std::max(max_dens, (a1 - a0) / vol);
    }
    e.n_chunks = (int)clo.size();
    if (cfg->max_neighbors > 0) {
        e.max_nb = cfg->max_neighbors;
    } else {
        double est = max_dens * 4.0 / 3.0 * M_PI * rl * rl * rl;
        int m = (int)std::ceil(1.4 * est + 24.0);
        m = (m + 7) / 8 * 8;
        e.max_nb = (int)std::max<int64_t>(8, std::min<int64_t>(m, std::max<int64_t>(max_box - 1, 1)));
    }

    int rc = MD_OK;
    size_t Np = (size_t)e.N_pad;
    size_t nk = knot_count(*pot);
#define AL(p, n) \
    if ((rc = dalloc(E, &(p), (n))) != MD_OK) goto fail_alloc;
    AL(e.L, 3 * B);
    AL(e.cell_len, 3 * B);
    AL(e.cell_len_f, 3 * B);
    AL(e.nc, 3 * B);
    AL(e.cell_off, B + 1);
    AL(e.atom_off, B + 1);
    AL(e.atom_box, e.N);
    AL(e.cell_box, tot);
    AL(e.cell_rank, tot);
    AL(e.cell_xyz, tot);
    AL(e.cell_org, tot);
    if (pot->kind == MD_POT_SPLINE) {
        AL(e.spline_coef, nk);
        AL(e.spline_coef_f, nk);
        if (pot->n_phi == pot->n_f) AL(e.spline_pair_rec, (size_t)pot_pairs(*pot) * (pot->n_phi + 1) * 4);
        AL(e.spline_work, 3 * nk);
        AL(e.knots_dev, nk);
    }
    AL(e.chunk_lo, e.n_chunks);
    AL(e.chunk_hi, e.n_chunks);
    AL(e.box_chunk_off, B + 1);
    AL(e.x, Np);
    AL(e.x_alt, Np);
    AL(e.xb, Np);
    AL(e.v, 3 * Np);
    AL(e.v_alt, 3 * Np);
    AL(e.f, 3 * Np);
    AL(e.rho, Np);
    AL(e.Fp, Np);
    AL(e.xf, Np);
    AL(e.e_atom, Np);
    AL(e.xo, Np);
    AL(e.xq, Np);
    AL(e.sum_q, kSumWords * Np);
    AL(e.perm, Np);
    AL(e.perm_alt, Np);
    AL(e.iperm, Np);
    AL(e.cell_of, Np);
    AL(e.cell_t, Np);
    AL(e.cell_t_alt, Np);
    AL(e.src, Np);
    AL(e.cell_count, tot);
    AL(e.cell_start, tot + 1);
    AL(e.scan_tmp, tot / 1024 + 2);
    AL(e.nn, Np);
    AL(e.nl, (size_t)e.max_nb * Np);
    if (cfg->precision == MD_FP64) {
        AL(e.pc, (size_t)e.max_nb * Np);
        AL(e.rev, (size_t)e.max_nb * Np);
        AL(e.nl_lo, (size_t)e.max_nb * Np);
        AL(e.n_up, Np);
    }
    AL(e.exp_T, kExpTable);
    if (pot->kind == MD_POT_RGL) {
        // the r table for this cutoff (a later potential may not raise it)
        const double rcut = pot->r_cut;
        AL(e.rx_tab, (size_t)(std::ceil(rcut * kRxPerA) + 2 - std::floor(0.3 * rcut * kRxPerA)));
    }
    AL(e.stage, 3 * std::max<size_t>(e.N, 1));
    AL(e.red, 2 * std::max(e.n_chunks, 1));
    AL(e.thermo_dev, 4 * (B + 1));
    AL(e.ctl, 1);
    AL(e.disp_box, B);
    AL(e.types, std::max<size_t>(Np, 1));
    AL(e.due_cells, tot);
#undef AL
    if (cudaMallocHost((void**)&e.ctl_host, sizeof(Ctl)) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(E, MD_ERR_NOMEM, "cudaMallocHost failed");
        goto fail_alloc;
    }
    {
        cudaStream_t s = nullptr;
        auto up = [&](void* d, const void* hsrc, size_t bytes) {
            return cudaMemcpy(d, hsrc, bytes, cudaMemcpyHostToDevice);
        };
        cudaError_t ce = cudaSuccess;
        ce = ce != cudaSuccess ? ce : up(e.L, box, 3 * B * sizeof(double));
        ce = ce != cudaSuccess ? ce : cudaMemset(e.types, 0, sizeof(int) * std::max<size_t>(Np, 1));
        ce = ce != cudaSuccess ? ce : up(e.cell_len, cl.data(), 3 * B * sizeof(double));
        ce = ce != cudaSuccess ? ce : up(e.cell_len_f, clf.data(), 3 * B * sizeof(float));
        ce = ce != cudaSuccess ? ce : up(e.nc, e.nc_h.data(), 3 * B * sizeof(int));
        ce = ce != cudaSuccess ? ce : up(e.cell_off, e.cell_off_h.data(), (B + 1) * sizeof(int));
        ce = ce != cudaSuccess ? ce : up(e.atom_off, atom_off, (B + 1) * sizeof(int64_t));
        if (e.N) ce = ce != cudaSuccess ? ce : up(e.atom_box, abox.data(), e.N * sizeof(int));
        ce = ce != cudaSuccess ? ce : up(e.cell_box, cbox.data(), tot * sizeof(int));
        ce = ce != cudaSuccess ? ce : up(e.cell_rank, rank.data(), tot * sizeof(int));
        ce = ce != cudaSuccess ? ce : up(e.cell_xyz, xyz.data(), tot * sizeof(int));
        {
            std::vector<double4_32a> org(tot);
            for (int c = 0; c < tot; ++c) {
                const int b = cbox[c], v = xyz[c];
                const int cc[3] = {v & 1023, (v >> 10) & 1023, (v >> 20) & 1023};
                double o[3];
                for (int a = 0; a < 3; ++a) o[a] = cc[a] * cl[3 * b + a];
                long long w = v;
                double wd;
                memcpy(&wd, &w, sizeof(wd));
                org[c] = make_double4_32a(o[0], o[1], o[2], wd);
            }
            ce = ce != cudaSuccess ? ce : up(e.cell_org, org.data(), tot * sizeof(double4_32a));
        }
        if (e.n_chunks) {
            ce = ce != cudaSuccess ? ce : up(e.chunk_lo, clo.data(), clo.size() * sizeof(int64_t));
            ce = ce != cudaSuccess ? ce : up(e.chunk_hi, chi.data(), chi.size() * sizeof(int64_t));
        }
        ce = ce != cudaSuccess ? ce : up(e.box_chunk_off, bco.data(), (B + 1) * sizeof(int));
        {
            // exponential table and reduction constants (long-double host arithmetic)
            std::vector<double> T(kExpTable);
            for (int j = 0; j < kExpTable; ++j) T[j] = (double)exp2l((long double)j / kExpTable);
            long double ln2 = logl(2.0L);
            e.exp_const.inv_l = (double)((long double)kExpTable / ln2);
            e.exp_const.l1 = (double)(ln2 / kExpTable);
            e.exp_const.l2 = (double)(ln2 / kExpTable - (long double)e.exp_const.l1);
            ce = ce != cudaSuccess ? ce : up(e.exp_T, T.data(), kExpTable * sizeof(double));
        }
        if (ce == cudaSuccess) ce = cudaMemset(e.cell_count, 0, tot * sizeof(int));
        if (ce == cudaSuccess) ce = cudaMemset(e.v, 0, 3 * Np * sizeof(double));
        if (ce == cudaSuccess) ce = cudaMemset(e.f, 0, 3 * Np * sizeof(double));
        if (ce == cudaSuccess) ce = cudaMemset(e.e_atom, 0, Np * sizeof(double));
        if (ce == cudaSuccess) ce = cudaMemset(e.sum_q, 0, kSumWords * Np * sizeof(long long));
        if (ce == cudaSuccess) ce = cudaMemset(e.ctl, 0, sizeof(Ctl));
        if (ce == cudaSuccess) ce = cudaMemset(e.disp_box, 0, sizeof(unsigned long long) * B);
        if (ce != cudaSuccess) {
            rc = fail(E, MD_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(ce));
            goto fail_alloc;
        }
        launch_reset_perm(e, s);
        if ((rc = upload_potential(h, s)) != MD_OK) goto fail_alloc;
        ce = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
        if (ce != cudaSuccess) {
            rc = fail(E, MD_ERR_CUDA, std::string("setup: ") + cudaGetErrorString(ce));
            goto fail_alloc;
        }
    }
    *out = h;
    return MD_OK;
fail_alloc:
    g_err = e.err;
    free_engine(e);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->body_stream) cudaStreamDestroy(h->body_stream);
    delete h;
    return rc;
}

// ---- transfers ----

// Device pointer for an input array: the array itself if it lives on the
// device, else a copy in the staging buffer.
// Host inputs go through the device stage with one bulk copy: kernels that
// read mapped page-locked memory in place (over the host link, in the
// library's sorted order) measured 1.35-1.9x slower end to end.
int stage_in(Engine* E, const double* src, size_t count, cudaStream_t s, const double** out) {
    if (is_device_ptr(src)) {
        *out = src;
        return MD_OK;
    }
    CK(cudaMemcpyAsync(E->stage, src, count * sizeof(double), cudaMemcpyHostToDevice, s));
    *out = E->stage;
    return MD_OK;
}

struct OutDst {
    double* dev;     // where the kernel writes
    double* host;    // host destination or NULL
    size_t count;
};

OutDst out_dst(Engine& e, double* dst, size_t count) {
    if (is_device_ptr(dst)) return {dst, nullptr, count};
    return {e.stage, dst, count};
}

int out_finish(Engine* E, const OutDst& o, cudaStream_t s) {
    if (o.host) CK(cudaMemcpyAsync(o.host, o.dev, o.count * sizeof(double), cudaMemcpyDeviceToHost, s));
    return MD_OK;
}

int read_ctl(Engine* E, cudaStream_t s) {
    CK(cudaMemcpyAsync(E->ctl_host, E->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // launches counted for captured rebuild bodies that the gate skipped
    const unsigned long long sk = E->ctl_host->n_gate_skip;
    E->launches -= (long long)(sk - E->gate_skip_seen) * E->graph_body_kernels;
    E->gate_skip_seen = sk;
    return MD_OK;
}

int clear_status(Engine* E, cudaStream_t s) {
    CK(cudaMemsetAsync(&E->ctl->status, 0, sizeof(int), s));
    CK(cudaMemsetAsync(&E->ctl->overflow_count, 0, sizeof(int), s));
    return MD_OK;
}

int grow_list(Engine* E, int needed) {
    Engine& e = *E;
    int m = std::max(needed + needed / 4 + 8, e.max_nb + e.max_nb / 2);
    m = (m + 7) / 8 * 8;
    int* nl = nullptr;
    if (dalloc(E, &nl, (size_t)m * e.N_pad) != MD_OK) return MD_ERR_NOMEM;
    if (e.pc) {
        double4_32a* pc = nullptr;
        int *rev = nullptr, *nl_lo = nullptr;
        if (dalloc(E, &pc, (size_t)m * e.N_pad) != MD_OK || dalloc(E, &rev, (size_t)m * e.N_pad) != MD_OK ||
            dalloc(E, &nl_lo, (size_t)m * e.N_pad) != MD_OK) {
            cudaFree(nl);
            if (pc) cudaFree(pc);
            if (rev) cudaFree(rev);
            return MD_ERR_NOMEM;
        }
        cudaFree(e.pc);
        cudaFree(e.rev);
        cudaFree(e.nl_lo);
        e.pc = pc;
        e.rev = rev;
        e.nl_lo = nl_lo;
    }
    cudaFree(e.nl);
    e.nl = nl;
    e.max_nb = m;
    destroy_graphs(e);
    return MD_OK;
}

// After a launch sequence that may have overflowed the list: grow and
// rebuild (list only: cells and order are already done) up to 4 times.
int settle_overflow(Engine* E, cudaStream_t s, bool* had) {
    *had = false;
    for (int attempt = 0;; ++attempt) {
        int rc = read_ctl(E, s);
        if (rc) return rc;
        int st = E->ctl_host->status;
        if (st & kStNonFinite) return fail(E, MD_ERR_NONFINITE, "non-finite energy");
        if (!(st & kStOverflow)) return MD_OK;
        *had = true;
        if (attempt >= 4)
            return fail(E, MD_ERR_NEIGH_OVERFLOW,
                        "neighbour list overflow: " + std::to_string(E->ctl_host->overflow_count) + " > " +
                            std::to_string(E->max_nb));
        if ((rc = grow_list(E, E->ctl_host->overflow_count)) != MD_OK) return rc;
        if ((rc = clear_status(E, s)) != MD_OK) return rc;
        // a full rebuild (binning too), so the lists and the build
        // positions agree again whatever stage the failed build reached
        launch_rebuild(*E, 1, s);
        CK(cudaGetLastError());
    }
}

int rebuild_and_forces(Engine* E, cudaStream_t s) {
    launch_rebuild(*E, 1, s);
    CK(cudaGetLastError());
    bool had;
    int rc = settle_overflow(E, s, &had);
    if (rc) return rc;
    launch_forces(*E, 0, s);
    launch_thermo(*E, s);
    CK(cudaGetLastError());
    return MD_OK;
}

// Forces after a load that kept the lists: boxes whose atoms moved more
// than half the skin from their build positions are rebuilt.
int refresh_and_forces(Engine* E, cudaStream_t s) {
    launch_rebuild(*E, 0, s);
    CK(cudaGetLastError());
    bool had;
    int rc = settle_overflow(E, s, &had);
    if (rc) return rc;
    launch_forces(*E, 0, s);
    launch_thermo(*E, s);
    launch_after_load(*E, s);
    CK(cudaGetLastError());
    return MD_OK;
}

int finish_sync(Engine* E, cudaStream_t s) {
    int rc = read_ctl(E, s);
    if (rc) return rc;
    if (E->ctl_host->status & kStNonFinite) return fail(E, MD_ERR_NONFINITE, "non-finite energy");
    if (E->ctl_host->status & kStOverflow) return fail(E, MD_ERR_NEIGH_OVERFLOW, "neighbour list overflow");
    if (E->ctl_host->status & kStCellSide)
        return fail(E, MD_ERR_UNSUPPORTED, "pressure coupling would shrink a box below one list radius per cell");
    return MD_OK;
}

int set_positions(Engine* E, const double* x, const double* v, bool set_v, cudaStream_t s) {
    Engine& e = *E;
    if (e.N == 0) {
        e.have_state = true;
        return MD_OK;
    }
    const double* xd = nullptr;
    // lists built for earlier positions stay usable for new ones within
    // half the skin of the build positions (the rule the steps follow): a
    // load then rebuilds only the boxes that moved farther
    const bool keep = e.have_state && e.lists_ok;
    const bool had_forces = e.forces_ok;
    e.lists_ok = false;
    e.forces_ok = false;
    launch_reset_ctl(e, s);
    int rc = stage_in(E, x, 3 * (size_t)e.N, s, &xd);
    if (rc) return rc;
    if (keep)
        launch_load_positions_keep(e, xd, s);
    else
        launch_load_positions(e, xd, s);
    if (set_v) {
        const double* vd = nullptr;
        if (v && (rc = stage_in(E, v, 3 * (size_t)e.N, s, &vd))) return rc;
        launch_load_velocities(e, vd, s);
    }
    CK(cudaGetLastError());
    // non-finite inputs: report before any list is built from them
    if ((rc = read_ctl(E, s))) return rc;
    if (E->ctl_host->status & kStNonFinite) return fail(E, MD_ERR_NONFINITE, "non-finite position or velocity");
    if (keep && had_forces && E->ctl_host->pos_changed == 0) {
        // every position is the current one: lists and forces stay valid,
        // only the energies follow the new velocities
        launch_thermo(e, s);
        launch_after_load(e, s);
        CK(cudaGetLastError());
    } else if ((rc = keep ? refresh_and_forces(E, s) : rebuild_and_forces(E, s))) {
        return rc;
    }
    e.have_state = true;
    if ((rc = finish_sync(E, s))) return rc;
    e.lists_ok = true;
    e.forces_ok = true;
    return MD_OK;
}

// ---- stepping ----

// Forces, second half-kick, the pressure coupling of Eq. (5) when on, and
// the step's bookkeeping.
void finish_step(Engine& e, bool hist, cudaStream_t s) {
    launch_forces(e, 1, s, e.baro.on);
    if (e.baro.on) {
        launch_thermo(e, s);
        launch_pressure(e, true, s);
    }
    launch_end_step(e, hist ? 1 : 0, s);
}

void enqueue_step(Engine& e, bool hist, cudaStream_t s) {
    launch_kick_drift(e, s);
    launch_rebuild(e, 0, s);
    finish_step(e, hist, s);
}

// One captured step whose rebuild kernels sit in the body of a conditional
// node set by k_rebuild_gate. Returns the first CUDA error.
cudaError_t capture_step_cond(md_batch* h, bool hist, long long* body_kernels) {
    Engine& e = h->e;
    cudaStream_t cs = h->cap_stream;
    launch_kick_drift(e, cs);
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t ce = cudaStreamGetCaptureInfo(cs, &st, nullptr, &g, &deps, nullptr, &nd);
    if (ce != cudaSuccess) return ce;
    cudaGraphConditionalHandle hc;
    if ((ce = cudaGraphConditionalHandleCreate(&hc, g, 0, 0)) != cudaSuccess) return ce;
    launch_rebuild_gate(e, hc, cs);
    if ((ce = cudaStreamGetCaptureInfo(cs, &st, nullptr, &g, &deps, nullptr, &nd)) != cudaSuccess) return ce;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hc;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((ce = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p)) != cudaSuccess) return ce;
    cudaGraph_t body = p.conditional.phGraph_out[0];
    if ((ce = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return ce;
    if ((ce = cudaStreamBeginCaptureToGraph(h->body_stream, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return ce;
    const long long b0 = e.launches;
    launch_rebuild(e, 0, h->body_stream);
    *body_kernels = e.launches - b0;
    cudaGraph_t done = nullptr;
    if ((ce = cudaStreamEndCapture(h->body_stream, &done)) != cudaSuccess) return ce;
    finish_step(e, hist, cs);
    return cudaGetLastError();
}

// Captures `steps` steps; last_energy: the last one forms the pair-energy
// sums (every step does when it records its energy or couples the pressure).
int capture(md_batch* h, int steps, bool hist, bool last_energy, cudaGraphExec_t* out, long long* kernels) {
    Engine* E = &h->e;
    cudaGraph_t g = nullptr;
    long long before = E->launches;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t cc = cudaSuccess;
    // single boxes only: in a batch some box is due on most steps, and the
    // gate's launch and node cost more than the skipped bodies save
    // (measured 1-2% slower on 16 and 256 boxes; 3% faster on one 2048-atom box)
    const bool gate = !E->cond_off && E->B == 1;
    for (int k = 0; k < steps; ++k) {
        E->pair_energy = hist || E->baro.on || (last_energy && k == steps - 1);
        if (gate && cc == cudaSuccess)
            cc = capture_step_cond(h, hist, &E->graph_body_kernels);
        else
            enqueue_step(h->e, hist, h->cap_stream);
    }
    E->pair_energy = true;
    cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
    *kernels = E->launches - before;
    E->launches = before;
    if (gate && (cc != cudaSuccess || ce != cudaSuccess)) {
        // conditional nodes unavailable: capture plain steps instead
        cudaStreamCaptureStatus bs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(h->body_stream, &bs) == cudaSuccess && bs != cudaStreamCaptureStatusNone) {
            cudaGraph_t t = nullptr;
            cudaStreamEndCapture(h->body_stream, &t);
            if (t) cudaGraphDestroy(t);
        }
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        E->cond_off = true;
        E->graph_body_kernels = 0;
        return capture(h, steps, hist, last_energy, out, kernels);
    }
    if (ce != cudaSuccess) return fail(E, MD_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fail(E, MD_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(ce));
    return MD_OK;
}

constexpr int kGraphChunk = 8;

// n steps; only the last one forms the pair-energy sums unless every step
// records its energy or couples the pressure (graph replay: n - 1 steps as
// chunks and single steps, then the last step's own graph).
int enqueue_steps(md_batch* h, int n, bool hist, bool use_graph, cudaStream_t s) {
    Engine* E = &h->e;
    Engine& e = *E;
    if (n <= 0) return MD_OK;
    if (!use_graph || e.N == 0 || e.prof_timing) {
        for (int k = 0; k < n; ++k) {
            e.pair_energy = hist || e.baro.on || k == n - 1;
            enqueue_step(e, hist, s);
        }
        e.pair_energy = true;
        CK(cudaGetLastError());
        return MD_OK;
    }
    if (e.graph_hist != hist) destroy_graphs(e);
    e.graph_hist = hist;
    int rc;
    const int body = n - 1;
    if (body >= kGraphChunk && !e.graph_chunk &&
        (rc = capture(h, kGraphChunk, hist, false, &e.graph_chunk, &e.graph_chunk_kernels)))
        return rc;
    if (body % kGraphChunk && !e.graph_step &&
        (rc = capture(h, 1, hist, false, &e.graph_step, &e.graph_step_kernels)))
        return rc;
    if (!e.graph_last && (rc = capture(h, 1, hist, true, &e.graph_last, &e.graph_last_kernels))) return rc;
    for (int k = 0; k < body / kGraphChunk; ++k) {
        CK(cudaGraphLaunch(e.graph_chunk, s));
        e.launches += e.graph_chunk_kernels;
    }
    for (int k = 0; k < body % kGraphChunk; ++k) {
        CK(cudaGraphLaunch(e.graph_step, s));
        e.launches += e.graph_step_kernels;
    }
    CK(cudaGraphLaunch(e.graph_last, s));
    e.launches += e.graph_last_kernels;
    return MD_OK;
}

int ensure_hist(Engine* E, int n) {
    Engine& e = *E;
    if (e.hist_cap >= n) return MD_OK;
    dfree(e.hist);
    int cap = std::max(n, 1024);
    if (dalloc(E, &e.hist, 4 * (size_t)cap) != MD_OK) return MD_ERR_NOMEM;
    e.hist_cap = cap;
    destroy_graphs(e);
    return MD_OK;
}

int steps_impl(md_batch* h, int n, double* hist_out, bool use_graph, cudaStream_t s) {
    Engine* E = &h->e;
    Engine& e = *E;
    if (n < 0) return fail(E, MD_ERR_ARG, "n_steps must be >= 0");
    if (!e.have_state) return fail(E, MD_ERR_ARG, "no state: call set_state or compute_forces first");
    bool hist = hist_out != nullptr;
    int rc;
    if (hist && (rc = ensure_hist(E, n))) return rc;
    if ((rc = read_ctl(E, s))) return rc;
    long long step0 = e.ctl_host->step;
    long long target = step0 + n;
    int remaining = n;
    while (remaining > 0) {
        if ((rc = enqueue_steps(h, remaining, hist, use_graph, s))) return rc;
        if ((rc = read_ctl(E, s))) return rc;
        int st = e.ctl_host->status;
        if (st & kStNonFinite) return fail(E, MD_ERR_NONFINITE, "non-finite energy");
        if (st & kStCellSide)
            return fail(E, MD_ERR_UNSUPPORTED, "pressure coupling would shrink a box below one list radius per cell");
        if (st & kStOverflow) {
            // the step that overflowed has drifted and re-sorted; finish it
            bool had;
            if ((rc = settle_overflow(E, s, &had))) return rc;
            finish_step(e, hist, s);
            CK(cudaGetLastError());
            if ((rc = read_ctl(E, s))) return rc;
        }
        remaining = (int)(target - e.ctl_host->step);
    }
    launch_thermo(e, s);
    CK(cudaGetLastError());
    if (hist) {
        // rows step0 .. step0+n-1 of the ring
        OutDst o = out_dst(e, hist_out, 4 * (size_t)n);
        for (long long k = 0; k < n;) {
            long long r = (step0 + k) % e.hist_cap;
            long long len = std::min<long long>(n - k, e.hist_cap - r);
            CK(cudaMemcpyAsync(o.dev + 4 * k, e.hist + 4 * r, 4 * len * sizeof(double), cudaMemcpyDefault, s));
            k += len;
        }
        if ((rc = out_finish(E, o, s))) return rc;
    }
    return finish_sync(E, s);
}

int thermo_impl(md_batch* h, md_thermo* out, double* per_box, cudaStream_t s) {
    Engine* E = &h->e;
    Engine& e = *E;
    double t[4];
    CK(cudaMemcpyAsync(t, e.thermo_dev + 4 * e.B, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    int rc;
    if (per_box) {
        OutDst o = out_dst(e, per_box, 4 * (size_t)e.B);
        CK(cudaMemcpyAsync(o.dev, e.thermo_dev, 4 * e.B * sizeof(double), cudaMemcpyDefault, s));
        if ((rc = out_finish(E, o, s))) return rc;
    }
    if ((rc = read_ctl(E, s))) return rc;
    if (out) {
        out->ke = t[0];
        out->pe = t[1];
        out->etot = t[2];
        out->temperature = t[3];
        double d2;
        memcpy(&d2, &e.ctl_host->disp2_last, sizeof(d2));
        out->max_disp = std::sqrt(d2);
        out->n_rebuild = e.ctl_host->n_rebuild;
        out->step = e.ctl_host->step;
    }
    return MD_OK;
}

md_batch* H(const md_batch* p) { return const_cast<md_batch*>(p); }

// n steps of the block-per-box schedule, growing the list and relaunching
// from where each box stopped when a box overflows it.
int box_steps(md_batch* h, int n, cudaStream_t s) {
    Engine* E = &h->e;
    int rc;
    for (int attempt = 0;; ++attempt) {
        rc = launch_box_steps(*E, n, attempt == 0, s);
        if (rc) return fail(E, rc, "box schedule launch failed");
        if ((rc = read_ctl(E, s))) return rc;
        int st = E->ctl_host->status;
        if (st & kStNonFinite) return fail(E, MD_ERR_NONFINITE, "non-finite energy");
        if (!(st & kStOverflow)) break;
        if (attempt >= 4) return fail(E, MD_ERR_NEIGH_OVERFLOW, "neighbour list overflow (box schedule)");
        if ((rc = grow_list(E, E->ctl_host->overflow_count))) return rc;
        if ((rc = clear_status(E, s))) return rc;
    }
    launch_advance_steps(*E, n, s);
    launch_thermo(*E, s);
    CK(cudaGetLastError());
    return finish_sync(E, s);
}

}  // namespace

// ====================================================================== ABI

extern "C" {

int md_create(const md_config* cfg, const md_potential* pot, int64_t n_atoms, md_ctx** out) {
    if (!cfg) return fail(nullptr, MD_ERR_ARG, "config is NULL");
    if (n_atoms < 0) return fail(nullptr, MD_ERR_ARG, "n_atoms must be >= 0");
    int64_t off[2] = {0, n_atoms};
    return create_impl(cfg, pot, 1, off, cfg->box, out);
}

int md_batch_create(const md_config* cfg, const md_potential* pot, int n_boxes, const int64_t* atom_offsets,
                    const double* box_lengths, md_batch** out) {
    if (!atom_offsets || !box_lengths) return fail(nullptr, MD_ERR_ARG, "offsets or box lengths are NULL");
    return create_impl(cfg, pot, n_boxes, atom_offsets, box_lengths, out);
}

int md_destroy(md_ctx* h) {
    if (!h) return MD_ERR_ARG;
    cudaDeviceSynchronize();
    free_engine(h->e);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->body_stream) cudaStreamDestroy(h->body_stream);
    delete h;
    return MD_OK;
}

int md_batch_destroy(md_batch* b) { return md_destroy(b); }

int md_set_state(md_ctx* h, const double* x, const double* v, md_stream s) {
    if (!h) return MD_ERR_ARG;
    Engine* E = &h->e;
    if (h->e.N > 0 && !x) return fail(E, MD_ERR_ARG, "x is NULL");
    return set_positions(E, x, v, true, (cudaStream_t)s);
}

int md_batch_set_state(md_batch* b, const double* x, const double* v, md_stream s) { return md_set_state(b, x, v, s); }

int md_get_state(md_ctx* h, double* x, double* v, md_stream st) {
    if (!h) return MD_ERR_ARG;
    Engine* E = &h->e;
    Engine& e = *E;
    cudaStream_t s = (cudaStream_t)st;
    if (!e.have_state) return fail(E, MD_ERR_ARG, "no state");
    int rc;
    if (x && e.N) {
        OutDst o = out_dst(e, x, 3 * (size_t)e.N);
        launch_store_vec(e, nullptr, e.x, o.dev, s);
        if ((rc = out_finish(E, o, s))) return rc;
    }
    if (v && e.N) {
        OutDst o = out_dst(e, v, 3 * (size_t)e.N);
        launch_store_vec(e, e.v, nullptr, o.dev, s);
        if ((rc = out_finish(E, o, s))) return rc;
    }
    CK(cudaGetLastError());
    return finish_sync(E, s);
}

int md_batch_get_state(md_batch* b, double* x, double* v, md_stream s) { return md_get_state(b, x, v, s); }

int md_build_neighbors(md_ctx* h, md_stream st) {
    if (!h) return MD_ERR_ARG;
    Engine* E = &h->e;
    if (!E->have_state) return fail(E, MD_ERR_ARG, "no state");
    if (E->N == 0) return MD_OK;
    cudaStream_t s = (cudaStream_t)st;
    int rc = rebuild_and_forces(E, s);
    if (rc) return rc;
    return finish_sync(E, s);
}

int md_max_count(md_ctx* h, int32_t* out) {
    if (!h || !out) return MD_ERR_ARG;
    Engine* E = &h->e;
    int rc = read_ctl(E, nullptr);
    if (rc) return rc;
    *out = E->N ? E->ctl_host->max_count : 0;
    return MD_OK;
}

int md_get_neighbors(md_ctx* h, int32_t* nn, int32_t* nl, int32_t ld, md_stream st) {
    if (!h) return MD_ERR_ARG;
    Engine* E = &h->e;
    Engine& e = *E;
    cudaStream_t s = (cudaStream_t)st;
    if (!e.have_state) return fail(E, MD_ERR_ARG, "no state");
    if (e.N == 0) return MD_OK;
    if (!is_device_ptr(nn) || !is_device_ptr(nl)) return fail(E, MD_ERR_ARG, "nn and nl must be device pointers");
    int rc = read_ctl(E, s);
    if (rc) return rc;
    if (ld < e.ctl_host->max_count)
        return fail(E, MD_ERR_ARG, "ld " + std::to_string(ld) + " < largest count " +
                                       std::to_string(e.ctl_host->max_count));
    launch_get_neighbors(e, nn, nl, ld, s);
    CK(cudaGetLastError());
    return finish_sync(E, s);
}

static int emit_outputs(md_batch* h, double* f, double* e_atom, double* rho, cudaStream_t s) {
    Engine* E = &h->e;
    Engine& e = *E;
    int rc;
    if (e.N == 0) return MD_OK;
    if (f) {
        OutDst o = out_dst(e, f, 3 * (size_t)e.N);
        launch_store_vec(e, e.f, nullptr, o.dev, s);
        if ((rc = out_finish(E, o, s))) return rc;
    }
    if (e_atom) {
        OutDst o = out_dst(e, e_atom, (size_t)e.N);
        launch_store_scalar(e, e.e_atom, o.dev, s);
        if ((rc = out_finish(E, o, s))) return rc;
    }
    if (rho) {
        OutDst o = out_dst(e, rho, (size_t)e.N);
        launch_store_scalar(e, e.rho, o.dev, s);
        if ((rc = out_finish(E, o, s))) return rc;
    }
    CK(cudaGetLastError());
    return MD_OK;
}

int md_compute_forces(md_ctx* h, const double* x, double* f, double* e_atom, double* rho, double* e_total,
                      md_stream st) {
    if (!h) return MD_ERR_ARG;
    Engine* E = &h->e;
    cudaStream_t s = (cudaStream_t)st;
    if (E->N > 0 && !x) return fail(E, MD_ERR_ARG, "x is NULL");
    int rc = set_positions(E, x, nullptr, false, s);
    if (rc) return rc;
    if ((rc = emit_outputs(h, f, e_atom, rho, s))) return rc;
    if (e_total) {
        OutDst o = out_dst(*E, e_total, 1);
        CK(cudaMemcpyAsync(o.dev, E->thermo_dev + 4 * E->B + 1, sizeof(double), cudaMemcpyDefault, s));
        if ((rc = out_finish(E, o, s))) return rc;
    }
    return finish_sync(E, s);
}

int md_get_forces(md_ctx* h, double* f, double* e_atom, double* rho, md_stream st) {
    if (!h) return MD_ERR_ARG;
    Engine* E = &h->e;
    cudaStream_t s = (cudaStream_t)st;
    if (!E->have_state) return fail(E, MD_ERR_ARG, "no state");
    int rc = emit_outputs(h, f, e_atom, rho, s);
    if (rc) return rc;
    return E->deferred_status ? MD_OK : finish_sync(E, s);
}

int md_batch_compute_forces(md_batch* b, const double* x, double* f, double* e_box, md_stream st) {
    if (!b) return MD_ERR_ARG;
    Engine* E = &b->e;
    cudaStream_t s = (cudaStream_t)st;
    if (E->N > 0 && !x) return fail(E, MD_ERR_ARG, "x is NULL");
    int rc = set_positions(E, x, nullptr, false, s);
    if (rc) return rc;
    if ((rc = emit_outputs(b, f, nullptr, nullptr, s))) return rc;
    if (e_box) {
        OutDst o = out_dst(*E, e_box, (size_t)E->B);
        launch_box_energy(*E, o.dev, s);
        if ((rc = out_finish(E, o, s))) return rc;
    }
    return finish_sync(E, s);
}

int md_step(md_ctx* h, int n_steps, md_thermo* out, double* thermo_hist, int use_graph, md_stream st) {
    if (!h) return MD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)st;
    h->e.forces_ok = false;
    int rc = steps_impl(h, n_steps, thermo_hist, use_graph != 0, s);
    if (rc) {
        h->e.lists_ok = false;  // the next state load rebuilds everything
        return rc;
    }
    // the last force pass saw the final positions unless a box scaling followed it
    h->e.forces_ok = n_steps > 0 && !h->e.baro.on;
    if (out) return thermo_impl(h, out, nullptr, s);
    return MD_OK;
}

int md_get_thermo(md_ctx* h, md_thermo* out, md_stream st) {
    if (!h || !out) return MD_ERR_ARG;
    Engine* E = &h->e;
    cudaStream_t s = (cudaStream_t)st;
    if (!E->have_state) return fail(E, MD_ERR_ARG, "no state");
    launch_thermo(*E, s);
    CK(cudaGetLastError());
    return thermo_impl(h, out, nullptr, s);
}

int md_batch_step(md_batch* b, int n_steps, int schedule, int use_graph, double* thermo_box, md_stream st) {
    if (!b) return MD_ERR_ARG;
    Engine* E = &b->e;
    cudaStream_t s = (cudaStream_t)st;
    if (schedule < MD_SCHED_AUTO || schedule > MD_SCHED_TILE) return fail(E, MD_ERR_ARG, "unknown schedule");
    int rc;
    if (!E->have_state) return fail(E, MD_ERR_ARG, "no state");
    if (n_steps < 0) return fail(E, MD_ERR_ARG, "n_steps must be >= 0");
    if (schedule == MD_SCHED_BOX && !box_schedule_fits(*E))
        return fail(E, MD_ERR_UNSUPPORTED, "the box schedule needs float64 and boxes that fit in shared memory");
    int remaining = n_steps;
    if (schedule == MD_SCHED_AUTO && E->sched_choice == 0) {
        if (!box_schedule_fits(*E)) {
            E->sched_choice = MD_SCHED_TILE;
        } else if (remaining >= 8) {
            // autotune on the first steps of the run: 4 steps each way, keep
            // the faster per step (both schedules give the same bits)
            float t_tile = 0.f, t_box = 0.f;
            cudaEvent_t a, c;
            CK(cudaEventCreate(&a));
            CK(cudaEventCreate(&c));
            CK(cudaEventRecord(a, s));
            if ((rc = steps_impl(b, 4, nullptr, use_graph != 0, s))) {
                E->lists_ok = false;
                return rc;
            }
            CK(cudaEventRecord(c, s));
            CK(cudaEventSynchronize(c));
            CK(cudaEventElapsedTime(&t_tile, a, c));
            CK(cudaEventRecord(a, s));
            if ((rc = box_steps(b, 4, s))) {
                E->lists_ok = false;
                return rc;
            }
            CK(cudaEventRecord(c, s));
            CK(cudaEventSynchronize(c));
            CK(cudaEventElapsedTime(&t_box, a, c));
            cudaEventDestroy(a);
            cudaEventDestroy(c);
            E->sched_choice = t_box < t_tile ? MD_SCHED_BOX : MD_SCHED_TILE;
            E->sched_ms[0] = t_tile / 4;
            E->sched_ms[1] = t_box / 4;
            remaining -= 8;
        }
    }
    bool box = schedule == MD_SCHED_BOX || (schedule == MD_SCHED_AUTO && E->sched_choice == MD_SCHED_BOX);
    E->forces_ok = false;
    rc = box ? box_steps(b, remaining, s) : steps_impl(b, remaining, nullptr, use_graph != 0, s);
    if (rc) {
        E->lists_ok = false;  // the next state load rebuilds everything
        return rc;
    }
    E->forces_ok = !box && remaining > 0 && !E->baro.on;
    if (thermo_box) return thermo_impl(b, nullptr, thermo_box, s);
    return MD_OK;
}

int md_batch_thermo(md_batch* b, double* thermo_box, md_stream st) {
    if (!b || !thermo_box) return MD_ERR_ARG;
    Engine* E = &b->e;
    cudaStream_t s = (cudaStream_t)st;
    if (!E->have_state) return fail(E, MD_ERR_ARG, "no state");
    launch_thermo(*E, s);
    CK(cudaGetLastError());
    if (E->deferred_status) {
        // the per-box records only (a host destination is complete on return)
        OutDst o = out_dst(*E, thermo_box, 4 * (size_t)E->B);
        CK(cudaMemcpyAsync(o.dev, E->thermo_dev, 4 * E->B * sizeof(double), cudaMemcpyDefault, s));
        return out_finish(E, o, s);
    }
    int rc = thermo_impl(b, nullptr, thermo_box, s);
    if (rc) return rc;
    return finish_sync(E, s);
}

int md_batch_schedule(const md_batch* b, int* choice, double* ms_tile, double* ms_box) {
    if (!b) return MD_ERR_ARG;
    if (choice) *choice = b->e.sched_choice;
    if (ms_tile) *ms_tile = b->e.sched_ms[0];
    if (ms_box) *ms_box = b->e.sched_ms[1];
    return MD_OK;
}

int md_set_thermostat(md_batch* b, double T_e, double tau_T) {
    if (!b) return MD_ERR_ARG;
    Engine* E = &b->e;
    if (!(T_e >= 0.0) || !std::isfinite(T_e)) return fail(E, MD_ERR_ARG, "T_e must be >= 0 and finite");
    if (!std::isfinite(tau_T)) return fail(E, MD_ERR_ARG, "tau_T must be finite");
    Bath bath{};
    bath.on = tau_T > 0.0;
    bath.T_e = T_e;
    bath.decay = bath.on ? exp(-E->cfg.dt / tau_T) : 1.0;  // exp(-2 (dt/2) / tau_T)
    bath.m_3kb = E->cfg.mass * kMVV / (3.0 * kBoltz);
    E->bath = bath;
    destroy_graphs(*E);  // captured launches carry the old parameters
    return MD_OK;
}

int md_set_newton3(md_batch* b, int on) {
    if (!b) return MD_ERR_ARG;
    Engine* E = &b->e;
    E->forces_ok = false;  // a later state load recomputes the forces
    if (on && E->cfg.precision != MD_FP64) return fail(E, MD_ERR_UNSUPPORTED, "Newton's third law variant is float64 only");
    E->newton3 = on != 0;
    destroy_graphs(*E);  // captured launches are those of the other variant
    return MD_OK;
}

static int ensure_pressure(Engine* E) {
    Engine& e = *E;
    if (e.w_atom) return MD_OK;
    if (dalloc(E, &e.w_atom, (size_t)e.N_pad) || dalloc(E, &e.red_w, (size_t)std::max(e.n_chunks, 1)) ||
        dalloc(E, &e.press_box, (size_t)e.B) || dalloc(E, &e.mu_box, (size_t)e.B))
        return fail(E, MD_ERR_NOMEM, "cudaMalloc failed");
    return MD_OK;
}

int md_set_barostat(md_batch* b, double P0, double tau_p, double beta) {
    if (!b) return MD_ERR_ARG;
    Engine* E = &b->e;
    E->forces_ok = false;  // a later state load recomputes the forces
    if (!std::isfinite(P0) || !std::isfinite(tau_p) || !std::isfinite(beta))
        return fail(E, MD_ERR_ARG, "P0, tau_p and beta must be finite");
    if (tau_p > 0.0 && !(beta > 0.0)) return fail(E, MD_ERR_ARG, "beta must be > 0");
    int rc = ensure_pressure(E);
    if (rc) return rc;
    Baro baro{};
    baro.on = tau_p > 0.0;
    baro.P0 = P0;
    baro.k = baro.on ? beta * (E->cfg.dt / tau_p) : 0.0;
    if (E->baro.on && !baro.on && E->N) {
        // the single-box kernels take the box from the host copy again
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(E->L_h.data(), E->L, sizeof(double) * 3 * E->B, cudaMemcpyDeviceToHost));
    }
    E->baro = baro;
    destroy_graphs(*E);  // captured steps carry the old sequence
    return MD_OK;
}

int md_set_types(md_batch* b, const int32_t* types, md_stream st) {
    if (!b) return MD_ERR_ARG;
    Engine* E = &b->e;
    E->forces_ok = false;  // a later state load recomputes the forces
    Engine& e = *E;
    cudaStream_t s = (cudaStream_t)st;
    if (e.N && !types) return fail(E, MD_ERR_ARG, "types is NULL");
    if (!e.N) return MD_OK;
    const int T = pot_types(e.pot_host);
    std::vector<int32_t> h((size_t)e.N);
    if (is_device_ptr(types)) {
        CK(cudaMemcpyAsync(h.data(), types, sizeof(int32_t) * e.N, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        std::copy(types, types + e.N, h.begin());
    }
    for (int64_t k = 0; k < e.N; ++k)
        if (h[k] < 0 || h[k] >= T) return fail(E, MD_ERR_ARG, "type out of range for the potential's species");
    CK(cudaMemcpyAsync(e.types, h.data(), sizeof(int32_t) * e.N, cudaMemcpyHostToDevice, s));
    if (e.have_state) {
        launch_apply_types(e, s);
        launch_forces(e, 0, s);
        launch_thermo(e, s);
        CK(cudaGetLastError());
        return finish_sync(E, s);
    }
    CK(cudaStreamSynchronize(s));
    return MD_OK;
}

int md_pressure(md_batch* b, double* p_box, md_stream st) {
    if (!b) return MD_ERR_ARG;
    Engine* E = &b->e;
    Engine& e = *E;
    cudaStream_t s = (cudaStream_t)st;
    if (!e.have_state) return fail(E, MD_ERR_ARG, "no state");
    if (!p_box) return fail(E, MD_ERR_ARG, "p_box is NULL");
    int rc = ensure_pressure(E);
    if (rc) return rc;
    if (e.N) {
        launch_forces(e, 0, s, true);  // the same forces, with the virial
        launch_thermo(e, s);
        launch_pressure(e, false, s);
        CK(cudaGetLastError());
        OutDst o = out_dst(e, p_box, (size_t)e.B);
        CK(cudaMemcpyAsync(o.dev, e.press_box, sizeof(double) * e.B, cudaMemcpyDefault, s));
        if ((rc = out_finish(E, o, s))) return rc;
    } else {
        std::vector<double> z(e.B, 0.0);
        if (is_device_ptr(p_box))
            CK(cudaMemcpyAsync(p_box, z.data(), sizeof(double) * e.B, cudaMemcpyHostToDevice, s));
        else
            std::copy(z.begin(), z.end(), p_box);
    }
    return finish_sync(E, s);
}

int md_get_box(md_batch* b, double* lengths, md_stream st) {
    if (!b) return MD_ERR_ARG;
    Engine* E = &b->e;
    if (!lengths) return fail(E, MD_ERR_ARG, "lengths is NULL");
    cudaStream_t s = (cudaStream_t)st;
    CK(cudaMemcpyAsync(lengths, E->L, sizeof(double) * 3 * E->B, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return MD_OK;
}

int md_batch_set_potential(md_batch* b, const md_potential* pot, md_stream st) {
    if (!b) return MD_ERR_ARG;
    Engine* E = &b->e;
    E->forces_ok = false;  // a later state load recomputes the forces
    cudaStream_t s = (cudaStream_t)st;
    std::string why;
    if (check_potential(pot, why) != MD_OK) return fail(E, MD_ERR_ARG, why);
    const md_potential& o = E->pot_host;
    if (pot->kind != o.kind) return fail(E, MD_ERR_ARG, "potential kind differs");
    if (pot->kind == MD_POT_SPLINE &&
        (pot->n_phi != o.n_phi || pot->n_f != o.n_f || pot->n_F != o.n_F || pot->r_lo != o.r_lo ||
         pot->r_hi != o.r_hi || pot_types(*pot) != pot_types(o)))
        return fail(E, MD_ERR_ARG, "spline knot counts or range differ");
    if (pot_cutoff(pot) > pot_cutoff(&o)) return fail(E, MD_ERR_ARG, "cutoff may not grow");
    E->pot_host = *pot;
    if (pot->kind == MD_POT_SPLINE) {
        size_t nk = knot_count(*pot);
        E->knots_host.assign(pot->knots, pot->knots + nk);
        E->pot_host.knots = nullptr;
    }
    destroy_graphs(*E);
    int rc = upload_potential(b, s);
    if (rc) return rc;
    if (E->have_state && E->N) {
        launch_forces(*E, 0, s);
        launch_thermo(*E, s);
        CK(cudaGetLastError());
    }
    int rc2 = E->deferred_status ? MD_OK : finish_sync(E, s);
    // the forces (and the pair cache) are those of the stored positions and
    // the new potential
    if (rc2 == MD_OK && E->have_state) E->forces_ok = true;
    return rc2;
}

int md_set_deferred_status(md_batch* b, int on) {
    if (!b) return MD_ERR_ARG;
    b->e.deferred_status = on != 0;
    return MD_OK;
}

int md_sync(md_batch* b, md_stream st) {
    if (!b) return MD_ERR_ARG;
    return finish_sync(&b->e, (cudaStream_t)st);
}

int md_param_grad(md_batch* b, const double* g_f, const double* g_e, double* grad, md_stream st) {
    if (!b) return MD_ERR_ARG;
    Engine* E = &b->e;
    cudaStream_t s = (cudaStream_t)st;
    if (!E->have_state) return fail(E, MD_ERR_ARG, "no state");
    // the adjoint reads the forward pass's values when they are current and
    // leaves them so; otherwise it rewrites rho and F'
    const bool keep = E->forces_ok && !E->newton3;
    if (E->pot_host.kind == MD_POT_SC) return fail(E, MD_ERR_UNSUPPORTED, "no gradient for Sutton-Chen");
    if (!grad || !is_device_ptr(grad)) return fail(E, MD_ERR_ARG, "grad must be a device pointer");
    if (E->N && (!g_f || !is_device_ptr(g_f))) return fail(E, MD_ERR_ARG, "g_f must be a device pointer");
    if (g_e && !is_device_ptr(g_e)) return fail(E, MD_ERR_ARG, "g_e must be a device pointer");
    Engine& e = *E;
    if (!e.grad_g && e.N > 0) {
        int nb = (int)((e.N + 127) / 128);
        e.grad_blocks = std::max(1, std::min(nb, 4 * e.n_sm));
        const md_potential& p = e.pot_host;
        // spline coefficients: 4 per interval of every table
        size_t ncoef = p.kind == MD_POT_SPLINE ? 4 * (knot_count(p) - 2 * pot_pairs(p) - pot_types(p)) : 5;
        if (dalloc(E, &e.grad_g, 3 * (size_t)e.N_pad) || dalloc(E, &e.grad_u, (size_t)e.N_pad) ||
            dalloc(E, &e.grad_Fpp, (size_t)e.N_pad) || dalloc(E, &e.grad_partial, (size_t)e.grad_blocks * ncoef) ||
            dalloc(E, &e.grad_coef, ncoef))
            return MD_ERR_NOMEM;
    }
    int rc;
    {
        PhaseScope scope(e, MD_PHASE_GRAD, s);
        rc = launch_param_grad(*E, g_f, g_e, grad, s);
    }
    E->forces_ok = keep;
    if (rc) return fail(E, rc, "parameter gradient failed");
    CK(cudaGetLastError());
    return E->deferred_status ? MD_OK : finish_sync(E, s);
}

int md_num_params(const md_batch* b) {
    if (!b) return -1;
    const md_potential& p = b->e.pot_host;
    return p.kind == MD_POT_SPLINE ? (int)knot_count(p) : 5;
}

int md_eval_math(md_batch* h, int fn, const double* x, int64_t n, double* out, md_stream st) {
    if (!h) return MD_ERR_ARG;
    Engine* E = &h->e;
    if (fn < 0 || fn > 5) return fail(E, MD_ERR_ARG, "unknown function");
    if (n < 0) return fail(E, MD_ERR_ARG, "n must be >= 0");
    if (n > 0 && (!is_device_ptr(x) || !is_device_ptr(out))) return fail(E, MD_ERR_ARG, "x and out must be device pointers");
    launch_eval_math(*E, fn, x, n, out, (cudaStream_t)st);
    CK(cudaGetLastError());
    return MD_OK;
}

int md_profile_start(md_batch* h, int timing) {
    if (!h) return MD_ERR_ARG;
    h->e.launches = 0;
    h->e.ev_used = 0;
    h->e.prof_timing = timing != 0;
    return MD_OK;
}

int md_profile_read(md_batch* h, md_profile* out) {
    if (!h || !out) return MD_ERR_ARG;
    Engine* E = &h->e;
    CK(cudaDeviceSynchronize());
    memset(out, 0, sizeof(*out));
    out->launches = E->launches;
    for (size_t k = 0; k < E->ev_used; ++k) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, E->ev_pool[2 * k], E->ev_pool[2 * k + 1]));
        int ph = E->ev_phase[k];
        out->ms[ph] += ms;
        out->timed[ph] += 1;
    }
    return MD_OK;
}

const char* md_status_string(int st) {
    switch (st) {
        case MD_OK: return "ok";
        case MD_ERR_ARG: return "invalid argument";
        case MD_ERR_CUDA: return "CUDA error";
        case MD_ERR_NOMEM: return "out of device memory";
        case MD_ERR_NEIGH_OVERFLOW: return "neighbour list overflow";
        case MD_ERR_NONFINITE: return "non-finite energy or force";
        case MD_ERR_TIMEOUT: return "device wait timed out";
        case MD_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

const char* md_last_error(const md_batch* h) { return h ? H(h)->e.err.c_str() : g_err.c_str(); }

}  // extern "C"
