// Mixed-precision density and force passes.
//
// Positions, velocities and the integrator stay float64. For the pair math
// each atom carries a float32 offset from the origin of the cell it was
// binned into at the last list build (xo, refreshed after every drift), so
// a separation is
//     d = (c_j - c_i) * cell_side + (o_j - o_i)
// with the cell difference taken as a minimum image in whole cells (exact)
// and both offsets below one cell side plus the skin: the float32 rounding
// error of d is ~1e-7 of a cell side, not of the box length. V, rho and
// their derivatives are evaluated in float32 (hardware exp2 / rsqrt); the
// per-atom sums rho_i, F_i and the pair energy add each group of 16 list
// entries in plain float32 and combine the groups with compensated float32
// accumulation (Neumaier), and F(rho_i), F'(rho_i) are taken in float64.
// The paper's own precedent is float32 positions inside its neighbour-list
// kernel (Sec. 4).
#include "md_device.cuh"

namespace mdk {

constexpr int kMNT = 128;
// List entries whose partner data (offset, F') are loaded together before
// their pair math: more loads in flight per thread, the sums in the same
// order and groups (4 entries: the 4M-atom step 1.98 -> 1.74 ms, 2 entries:
// 1.92 ms; the compiler's float32 contractions may differ between batch
// sizes, so results differ by float32 rounding).
#ifndef MD_MIXED_BATCH
#define MD_MIXED_BATCH 4
#endif
constexpr int kMB = MD_MIXED_BATCH;

template <int KIND, bool SINGLE, bool WIDE>
__global__ void __launch_bounds__(kMNT) k_density_mixed(int64_t N, int64_t Np, Geo g, CellSep cs0, Pot P,
                                                        const float4* __restrict__ xo, const int* __restrict__ nn,
                                                        const int* __restrict__ nl, int max_nb,
                                                        double* __restrict__ rho, double* __restrict__ Fp,
                                                        float* __restrict__ Fpf, double* __restrict__ e_atom,
                                                        const Ctl* ctl) {
    if (load_status(ctl)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const CellSep cs = cell_sep<SINGLE>(g, cs0, i);
    const float4 oi = xo[i];
    const int n = min(nn[i], max_nb);
    GSum acc;
    for (int k0 = 0; k0 < n; k0 += kMB) {
        int eb[kMB];
        float4 ob[kMB];
#pragma unroll
        for (int u = 0; u < kMB; ++u) eb[u] = k0 + u < n ? nl[(int64_t)(k0 + u) * Np + i] : 0;
#pragma unroll
        for (int u = 0; u < kMB; ++u) ob[u] = k0 + u < n ? xo[entry_slot(eb[u])] : oi;
#pragma unroll
        for (int u = 0; u < kMB; ++u) {
            const int k = k0 + u;
            if (k >= n) break;
            float dx, dy, dz;
            sep_mixed_entry<WIDE>(cs, oi, ob[u], eb[u], dx, dy, dz);
            float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.f_rc2) acc.add(dens_ff<KIND>(P, r2 * rsqrtf(r2), species_pair<KIND>(P, oi, ob[u])));
            if ((k & kGroupMask) == kGroupMask) acc.flush();
        }
    }
    double r_i = acc.value();
    double F, Fpi;
    embed<KIND>(P, r_i, F, Fpi, KIND == MD_POT_SPLINE ? off_type(oi) : 0);
    rho[i] = r_i;
    Fp[i] = Fpi;
    Fpf[i] = (float)Fpi;
    e_atom[i] = F;
}

// Resident blocks per multiprocessor: with one entry in flight per thread
// the pass waits on gathered offsets and F', and 12 blocks (40 registers, a
// few spilled to L1) hid more of that than the spills cost (8% faster than
// 54 registers); with a batch of entries in flight the registers go to the
// batch instead.
#ifndef MD_MIXED_FORCE_BLOCKS
#define MD_MIXED_FORCE_BLOCKS (kMB == 1 ? 12 : 8)
#endif
template <int KIND, bool SINGLE, bool WIDE>
__global__ void __launch_bounds__(kMNT, MD_MIXED_FORCE_BLOCKS) k_force_mixed(int64_t N, int64_t Np, Geo g, CellSep cs0, Pot P,
                                                      const float4* __restrict__ xo, const int* __restrict__ nn,
                                                      const int* __restrict__ nl, int max_nb,
                                                      const float* __restrict__ Fpf, double* __restrict__ f,
                                                      double* __restrict__ e_atom, double* __restrict__ v,
                                                      double c_kick, Bath bath, double* __restrict__ w_atom,
                                                      const Ctl* ctl) {
    if (load_status(ctl)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const CellSep cs = cell_sep<SINGLE>(g, cs0, i);
    const float4 oi = xo[i];
    const float Fpi = Fpf[i];
    const int n = min(nn[i], max_nb);
    // w_atom (pressure users only): per-atom virial -1/2 sum_j s_ij r_ij^2
    const bool vir = w_atom != nullptr;
    GSum ax, ay, az, ae, aw;
    for (int k0 = 0; k0 < n; k0 += kMB) {
        int eb[kMB];
        float4 ob[kMB];
        float fb[kMB];
#pragma unroll
        for (int u = 0; u < kMB; ++u) eb[u] = k0 + u < n ? nl[(int64_t)(k0 + u) * Np + i] : 0;
#pragma unroll
        for (int u = 0; u < kMB; ++u) {
            const bool ok = k0 + u < n;
            ob[u] = ok ? xo[entry_slot(eb[u])] : oi;
            fb[u] = ok ? Fpf[entry_slot(eb[u])] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kMB; ++u) {
            const int k = k0 + u;
            if (k >= n) break;
            if ((k & kGroupMask) == 0 && k) {
                ax.flush();
                ay.flush();
                az.flush();
                ae.flush();
                if (vir) aw.flush();
            }
            float dx, dy, dz;
            sep_mixed_entry<WIDE>(cs, oi, ob[u], eb[u], dx, dy, dz);
            float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.f_rc2) {
                float rinv = rsqrtf(r2);
                float r = r2 * rinv;
                float phi, dphi, fr, dfr;
                pair_allf<KIND>(P, r, phi, dphi, fr, dfr, species_pair<KIND>(P, oi, ob[u]));
                float s = (dphi + (Fpi + fb[u]) * dfr) * rinv;
                ax.add(s * dx);
                ay.add(s * dy);
                az.add(s * dz);
                ae.add(phi);
                if (vir) aw.add(s * r2);
            }
        }
    }
    double fx = ax.value(), fy = ay.value(), fz = az.value();
    f[i] = fx;
    f[Np + i] = fy;
    f[2 * Np + i] = fz;
    e_atom[i] += 0.5 * ae.value();
    if (vir) w_atom[i] = -0.5 * aw.value();
    if (v) {
        double vx = v[i] + c_kick * fx, vy = v[Np + i] + c_kick * fy, vz = v[2 * Np + i] + c_kick * fz;
        bath_half(bath, vx, vy, vz);  // friction half step after the kick
        v[i] = vx;
        v[Np + i] = vy;
        v[2 * Np + i] = vz;
    }
}

CellSep single_cell_sep(const Engine& e) {
    CellSep cs{};
    if (e.B != 1) return cs;
    cs.lx = (float)(e.L_h[0] / e.nc_h[0]);
    cs.ly = (float)(e.L_h[1] / e.nc_h[1]);
    cs.lz = (float)(e.L_h[2] / e.nc_h[2]);
    cs.nx = e.nc_h[0];
    cs.ny = e.nc_h[1];
    cs.nz = e.nc_h[2];
    cs.Lx = (float)e.L_h[0];
    cs.Ly = (float)e.L_h[1];
    cs.Lz = (float)e.L_h[2];
    return cs;
}

template <int KIND, bool SINGLE, bool WIDE>
static void run_mixed(Engine& e, int kick, cudaStream_t s, bool virial) {
    Geo g = make_geo(e);
    const CellSep cs = single_cell_sep(e);
    int nb = (int)((e.N + kMNT - 1) / kMNT);
    double c_kick = 0.5 * e.cfg.dt / (e.cfg.mass * kMVV);
    e.launches += 2;
    {
        PhaseScope scope(e, MD_PHASE_DENSITY, s);
        k_density_mixed<KIND, SINGLE, WIDE><<<nb, kMNT, 0, s>>>(e.N, e.N_pad, g, cs, e.pot, e.xo, e.nn, e.nl, e.max_nb,
                                                         e.rho, e.Fp, e.Fpf, e.e_atom, e.ctl);
    }
    PhaseScope scope(e, MD_PHASE_FORCE, s);
    k_force_mixed<KIND, SINGLE, WIDE><<<nb, kMNT, 0, s>>>(e.N, e.N_pad, g, cs, e.pot, e.xo, e.nn, e.nl, e.max_nb, e.Fpf,
                                                   e.f, e.e_atom, kick ? e.v : nullptr, c_kick, e.bath,
                                                   virial ? e.w_atom : nullptr, e.ctl);
}

template <int KIND>
static void run_mixed_k(Engine& e, int kick, cudaStream_t s, bool virial) {
    if (single_fast(e))
        e.wide ? run_mixed<KIND, true, true>(e, kick, s, virial) : run_mixed<KIND, true, false>(e, kick, s, virial);
    else
        e.wide ? run_mixed<KIND, false, true>(e, kick, s, virial) : run_mixed<KIND, false, false>(e, kick, s, virial);
}

void launch_forces_mixed(Engine& e, int kick, cudaStream_t s, bool virial) {
    switch (e.pot.kind) {
        case MD_POT_RGL: run_mixed_k<MD_POT_RGL>(e, kick, s, virial); break;
        case MD_POT_SC: run_mixed_k<MD_POT_SC>(e, kick, s, virial); break;
        default: run_mixed_k<MD_POT_SPLINE>(e, kick, s, virial); break;
    }
}

}  // namespace mdk
