// Time integration, reductions and caller-order copies.
//
//   k_kick_drift   v += dt/2 F/m; x += dt v; largest displacement since
//                  the last list build (device rebuild trigger); refresh
//                  the cell-local float32 offsets (float32 screens and
//                  mixed-precision pair math)
//   k_end_step     step bookkeeping on the device (no host round trip)
//   k_chunk_sums / k_thermo_final
//                  deterministic fixed-order sums of kinetic and potential
//                  energy per box, totals, temperature, non-finite check
// The paper integrates with a predictor-corrector (Sec. 3.3); velocity
// Verlet replaces it here.
#include <algorithm>

#include "md_device.cuh"

namespace mdk {

constexpr int kINT = 256;

static int nblk(int64_t n, int nt) { return (int)((n + nt - 1) / nt); }

// Largest squared displacement per box into disp[] (non-negative doubles
// order like their bit patterns): one atomic per block when the block's
// atoms lie in one box, per lane where a box boundary falls inside it.
// b < 0 marks a thread without an atom. Every thread of the block calls it.
template <bool SINGLE>
__device__ __forceinline__ void record_disp(const Geo& g, int64_t N, int b, double d2,
                                            unsigned long long* __restrict__ disp) {
    __shared__ double sm[kINT / 32];
    __shared__ int s_b0, s_b1;
    if (threadIdx.x == 0) {
        int64_t f = (int64_t)blockIdx.x * blockDim.x, l = min(f + blockDim.x, N) - 1;
        s_b0 = SINGLE ? 0 : g.atom_box[f];
        s_b1 = SINGLE ? 0 : g.atom_box[l];
    }
    __syncthreads();
    if (s_b0 == s_b1) {
        d2 = warp_max(d2);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = d2;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int k = 0; k < kINT / 32; ++k) m = sm[k] > m ? sm[k] : m;
            if (m > 0.0) atomicMax(&disp[s_b0], (unsigned long long)__double_as_longlong(m));
        }
    } else if (b >= 0 && d2 > 0.0) {
        atomicMax(&disp[b], (unsigned long long)__double_as_longlong(d2));
    }
}

template <bool SINGLE>
__global__ void __launch_bounds__(kINT) k_kick_drift(int64_t N, int64_t Np, Geo g, double4_32a* __restrict__ x,
                                                     double* __restrict__ v, const double* __restrict__ f,
                                                     const double4_32a* __restrict__ xb, double c_kick, Bath bath,
                                                     double dt,
                                                     float4* __restrict__ xo, const int* __restrict__ cell_t,
                                                     Ctl* ctl, unsigned long long* __restrict__ disp) {
    if (load_status(ctl)) return;
    // one box: a grid-stride loop over a few waves of blocks, so that the
    // per-block displacement maxima meet in few atomics on the box's word
    // (one atomic per 256 atoms serialised on that one address); several
    // boxes: one atom per thread (a block's atoms span one or two boxes)
    double d2 = 0.0;
    int b = -1;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = SINGLE ? (int64_t)gridDim.x * blockDim.x : N;
    for (int64_t i = i0; i < N; i += stride) {
        b = SINGLE ? 0 : g.atom_box[i];
        double4_32a p = x[i];
        double4_32a q = xb[i];
        double vx = v[i], vy = v[Np + i], vz = v[2 * Np + i];
        bath_half(bath, vx, vy, vz);  // friction half step before the kick
        vx = vx + c_kick * f[i];
        vy = vy + c_kick * f[Np + i];
        vz = vz + c_kick * f[2 * Np + i];
        // no wrap here: positions stay continuous until the next list build
        // (which wraps them), so the image stored in each list entry holds
        p.x += dt * vx;
        p.y += dt * vy;
        p.z += dt * vz;
        v[i] = vx;
        v[Np + i] = vy;
        v[2 * Np + i] = vz;
        x[i] = p;
        double dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
        const double di = dx * dx + dy * dy + dz * dz;
        d2 = di > d2 ? di : d2;
        // offset from the origin of the atom's cell at the last build; it
        // may leave [0, cell side) by the drift since then, which every user
        // of the offsets allows for
        const double4_32a org = g.cell_org[cell_t[i]];
        xo[i] = make_float4((float)(p.x - org.x), (float)(p.y - org.y), (float)(p.z - org.z),
                            __int_as_float((int)__double_as_longlong(org.w) | (pos_type(p) << 30)));
    }
    record_disp<SINGLE>(g, N, b, d2, disp);
}

// Closes a step: records the largest displacement over boxes, clears the
// per-box displacement words and counts the step (one block, fixed order).
__global__ void __launch_bounds__(1024) k_end_step(Ctl* ctl, int B, unsigned long long* __restrict__ disp) {
    if (load_status(ctl)) return;
    __shared__ unsigned long long sm[32];
    unsigned long long m = 0ull;
    for (int b = threadIdx.x; b < B; b += 1024) {
        unsigned long long v = disp[b];
        m = v > m ? v : m;
        disp[b] = 0ull;
    }
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0ull;
        for (int k = 0; k < 32; ++k) t = sm[k] > t ? sm[k] : t;
        ctl->disp2_last = t;
        ctl->step += 1;
    }
}

__global__ void k_reset_ctl(Ctl* ctl, int B, unsigned long long* __restrict__ disp) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->status = 0;
        ctl->overflow_count = 0;
        ctl->disp2_last = 0ull;
        ctl->step = 0;
        ctl->n_rebuild = 0;
        ctl->pos_changed = 0;
    }
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) disp[b] = 0ull;
}

constexpr int kRNT = 256;

// partial sums over one chunk of atoms of one box: (sum v^2, sum E_i)
__global__ void __launch_bounds__(kRNT) k_chunk_sums(int64_t Np, const int64_t* __restrict__ lo,
                                                     const int64_t* __restrict__ hi, const double* __restrict__ v,
                                                     const double* __restrict__ e_atom, double* __restrict__ part) {
    __shared__ double sh[kRNT / 32];
    int c = blockIdx.x;
    int64_t a = lo[c], b = hi[c];
    double sv = 0.0, se = 0.0;
    for (int64_t i = a + threadIdx.x; i < b; i += kRNT) {
        double vx = v[i], vy = v[Np + i], vz = v[2 * Np + i];
        sv += vx * vx + vy * vy + vz * vz;
        se += e_atom[i];
    }
    double tv = block_sum<kRNT>(sv, sh);
    double te = block_sum<kRNT>(se, sh);
    if (threadIdx.x == 0) {
        part[2 * c] = tv;
        part[2 * c + 1] = te;
    }
}

// ---- pressure (Eq. 6) and its Berendsen coupling (Eq. 5)

// per-chunk sums of the per-atom virial, fixed order
__global__ void __launch_bounds__(kRNT) k_chunk_virial(const int64_t* __restrict__ lo, const int64_t* __restrict__ hi,
                                                       const double* __restrict__ w, double* __restrict__ part) {
    __shared__ double sh[kRNT / 32];
    const int c = blockIdx.x;
    double sw = 0.0;
    for (int64_t i = lo[c] + threadIdx.x; i < hi[c]; i += kRNT) sw += w[i];
    const double t = block_sum<kRNT>(sw, sh);
    if (threadIdx.x == 0) part[c] = t;
}

// Pressure of every box, P = (N k_B T + W/3)/V with T the box's kinetic
// temperature of the thermo pass; when coupled, the factor
// mu = [1 - beta (dt/tau_p)(P0 - P)]^(1/3). A box whose cells would fall
// below one list radius raises kStCellSide, and then no box is scaled.
__global__ void k_box_pressure(int B, const int* __restrict__ box_chunk_off, const int64_t* __restrict__ atom_off,
                               const double* __restrict__ part_w, const double* __restrict__ thermo,
                               const double* __restrict__ L, const int* __restrict__ nc, double rl, Baro baro,
                               double* __restrict__ press, double* __restrict__ mu, Ctl* ctl) {
    if (load_status(ctl)) return;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        double W = 0.0;
        for (int c = box_chunk_off[b]; c < box_chunk_off[b + 1]; ++c) W += part_w[c];
        const double n = (double)(atom_off[b + 1] - atom_off[b]);
        const double V = L[3 * b] * L[3 * b + 1] * L[3 * b + 2];
        const double P = (n * kBoltz * thermo[4 * b + 3] + W / 3.0) / V;
        press[b] = P;
        if (!baro.on) continue;
        double m = cbrt(1.0 - baro.k * (baro.P0 - P));
        bool ok = true;
        for (int a = 0; a < 3; ++a) ok = ok && L[3 * b + a] * m / nc[3 * b + a] >= rl;
        if (!ok) {
            atomicOr(&ctl->status, kStCellSide);
            m = 1.0;
        }
        mu[b] = m;
    }
}

// Applies the factors of k_box_pressure to the box and cell lengths (after
// every box passed the cell check, so either all boxes scale or none).
__global__ void k_scale_boxes(int B, const double* __restrict__ mu, double* __restrict__ L,
                              double* __restrict__ cell_len, float* __restrict__ cell_len_f, const Ctl* ctl) {
    if (load_status(ctl)) return;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const double m = mu[b];
        for (int a = 0; a < 3; ++a) {
            L[3 * b + a] *= m;
            cell_len[3 * b + a] *= m;
            cell_len_f[3 * b + a] = (float)cell_len[3 * b + a];
        }
    }
}

__global__ void k_scale_atoms(int64_t N, Geo g, const double* __restrict__ mu, double4_32a* __restrict__ x,
                              const Ctl* ctl) {
    if (load_status(ctl)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = mu[g.B == 1 ? 0 : g.atom_box[i]];
        double4_32a p = x[i];
        p.x *= m;
        p.y *= m;
        p.z *= m;
        x[i] = p;
    }
}

__global__ void k_scale_cells(int n_cells, Geo g, const double* __restrict__ mu, double4_32a* __restrict__ org,
                              const Ctl* ctl) {
    if (load_status(ctl)) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
        const double m = mu[g.cell_box[c]];
        double4_32a o = org[c];
        o.x *= m;
        o.y *= m;
        o.z *= m;
        org[c] = o;
    }
}

// per-box and total (ke, pe, etot, T); optional history row
__global__ void __launch_bounds__(1024) k_thermo_final(int B, const int* __restrict__ box_chunk_off,
                                                       const int64_t* __restrict__ atom_off,
                                                       const double* __restrict__ part, double half_mv,
                                                       double* __restrict__ thermo, double* __restrict__ hist,
                                                       int hist_cap, Ctl* ctl) {
    __shared__ double sh[32];
    double ke_t = 0.0, pe_t = 0.0, dof_t = 0.0;
    for (int b = threadIdx.x; b < B; b += 1024) {
        double sv = 0.0, se = 0.0;
        for (int c = box_chunk_off[b]; c < box_chunk_off[b + 1]; ++c) {
            sv += part[2 * c];
            se += part[2 * c + 1];
        }
        double ke = half_mv * sv;
        double nb = (double)(atom_off[b + 1] - atom_off[b]);
        double dof = 3.0 * nb - 3.0;
        thermo[4 * b] = ke;
        thermo[4 * b + 1] = se;
        thermo[4 * b + 2] = ke + se;
        thermo[4 * b + 3] = dof > 0.0 ? 2.0 * ke / (dof * kBoltz) : 0.0;
        ke_t += ke;
        pe_t += se;
        dof_t += dof > 0.0 ? dof : 0.0;
    }
    double ke = block_sum<1024>(ke_t, sh);
    double pe = block_sum<1024>(pe_t, sh);
    double dof = block_sum<1024>(dof_t, sh);
    if (threadIdx.x == 0) {
        double* t = thermo + 4 * B;
        t[0] = ke;
        t[1] = pe;
        t[2] = ke + pe;
        t[3] = dof > 0.0 ? 2.0 * ke / (dof * kBoltz) : 0.0;
        if (!isfinite(ke) || !isfinite(pe)) atomicOr(&ctl->status, kStNonFinite);
        if (hist) {
            long long s = ctl->step % hist_cap;
            for (int k = 0; k < 4; ++k) hist[4 * s + k] = t[k];
        }
    }
}

template <bool SINGLE>
static void kick_drift_t(Engine& e, cudaStream_t s) {
    Geo g = make_geo(e);
    int nb = (int)((e.N + kINT - 1) / kINT);
    if (SINGLE) nb = std::min(nb, 8 * e.n_sm);  // one wave of 8 resident blocks per SM, grid-stride
    double c_kick = 0.5 * e.cfg.dt / (e.cfg.mass * kMVV);
    PhaseScope scope(e, MD_PHASE_KICK_DRIFT, s);
    e.launches += 1;
    k_kick_drift<SINGLE><<<nb, kINT, 0, s>>>(e.N, e.N_pad, g, e.x, e.v, e.f, e.xb, c_kick, e.bath, e.cfg.dt, e.xo,
                                                   e.cell_t, e.ctl, e.disp_box);
}

void launch_kick_drift(Engine& e, cudaStream_t s) {
    if (e.N == 0) return;
    if (single_fast(e))
        kick_drift_t<true>(e, s);
    else
        kick_drift_t<false>(e, s);
}

void launch_pressure(Engine& e, bool couple, cudaStream_t s) {
    if (e.N == 0) return;
    PhaseScope scope(e, MD_PHASE_OTHER, s);
    Baro b = e.baro;
    b.on = couple && e.baro.on;
    e.launches += b.on ? 5 : 2;
    k_chunk_virial<<<e.n_chunks, kRNT, 0, s>>>(e.chunk_lo, e.chunk_hi, e.w_atom, e.red_w);
    k_box_pressure<<<std::max(1, std::min((e.B + 255) / 256, 64)), 256, 0, s>>>(
        e.B, e.box_chunk_off, e.atom_off, e.red_w, e.thermo_dev, e.L, e.nc, e.rl, b, e.press_box, e.mu_box, e.ctl);
    if (b.on) {
        Geo g = make_geo(e);
        k_scale_boxes<<<std::max(1, std::min((e.B + 255) / 256, 64)), 256, 0, s>>>(e.B, e.mu_box, e.L, e.cell_len,
                                                                                  e.cell_len_f, e.ctl);
        k_scale_atoms<<<(int)std::min<int64_t>(nblk(e.N, 256), (int64_t)8 * e.n_sm), 256, 0, s>>>(e.N, g, e.mu_box,
                                                                                                   e.x, e.ctl);
        k_scale_cells<<<std::max(1, std::min(nblk(e.n_cells, 256), 8 * e.n_sm)), 256, 0, s>>>(e.n_cells, g, e.mu_box,
                                                                                              e.cell_org, e.ctl);
    }
}

void launch_end_step(Engine& e, int record_hist, cudaStream_t s) {
    if (record_hist) launch_thermo_hist(e, s);
    PhaseScope scope(e, MD_PHASE_OTHER, s);
    e.launches += 1;
    k_end_step<<<1, 1024, 0, s>>>(e.ctl, e.B, e.disp_box);
}

static void thermo_impl(Engine& e, bool hist, cudaStream_t s) {
    PhaseScope scope(e, MD_PHASE_OTHER, s);
    e.launches += e.n_chunks > 0 ? 2 : 1;
    if (e.n_chunks > 0)
        k_chunk_sums<<<e.n_chunks, kRNT, 0, s>>>(e.N_pad, e.chunk_lo, e.chunk_hi, e.v, e.e_atom, e.red);
    double half_mv = 0.5 * e.cfg.mass * kMVV;
    k_thermo_final<<<1, 1024, 0, s>>>(e.B, e.box_chunk_off, e.atom_off, e.red, half_mv, e.thermo_dev,
                                      hist ? e.hist : nullptr, e.hist_cap, e.ctl);
}

void launch_thermo(Engine& e, cudaStream_t s) { thermo_impl(e, false, s); }
void launch_thermo_hist(Engine& e, cudaStream_t s) { thermo_impl(e, true, s); }

__global__ void k_advance_steps(Ctl* ctl, long long n) { ctl->step += n; }

void launch_advance_steps(Engine& e, long long n, cudaStream_t s) {
    e.launches += 1;
    k_advance_steps<<<1, 1, 0, s>>>(e.ctl, n);
}

void launch_reset_ctl(Engine& e, cudaStream_t s) {
    e.launches += 1;
    k_reset_ctl<<<(e.B + 255) / 256, 256, 0, s>>>(e.ctl, e.B, e.disp_box);
}

// ---------------------------------------------------------------- copies

__global__ void k_load_pos(int64_t N, const double* __restrict__ src, const int* __restrict__ iperm, Geo g,
                           const int* __restrict__ types, double4_32a* __restrict__ x, Ctl* ctl) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    if (!isfinite(src[3 * c]) || !isfinite(src[3 * c + 1]) || !isfinite(src[3 * c + 2]))
        atomicOr(&ctl->status, kStNonFinite);
    int b = g.B == 1 ? 0 : g.atom_box[c];
    int t = iperm[c];
    double4_32a p;
    p.x = wrap_coord(src[3 * c], g.L[3 * b]);
    p.y = wrap_coord(src[3 * c + 1], g.L[3 * b + 1]);
    p.z = wrap_coord(src[3 * c + 2], g.L[3 * b + 2]);
    p.w = (double)types[c];  // the species rides in the pad lane
    x[t] = p;
}

// Positions for a handle whose lists stay usable: each caller position is
// wrapped and, where the atom crossed a face since the last build, moved to
// the image next to its build position (positions stay continuous between
// builds, as the image codes of the list entries require); otherwise the
// caller's value is kept as is. The displacement from the build position
// feeds the per-box rebuild decision, and the float32 offsets are refreshed.
template <bool SINGLE>
__global__ void __launch_bounds__(kINT) k_load_pos_keep(int64_t N, const double* __restrict__ src,
                                                        const int* __restrict__ iperm, Geo g,
                                                        double4_32a* __restrict__ x,
                                                        const double4_32a* __restrict__ xb, float4* __restrict__ xo,
                                                        const int* __restrict__ cell_t, const int* __restrict__ types,
                                                        Ctl* ctl, unsigned long long* __restrict__ disp) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0;
    int b = -1;
    bool changed = false;
    if (c < N) {
        if (!isfinite(src[3 * c]) || !isfinite(src[3 * c + 1]) || !isfinite(src[3 * c + 2]))
            atomicOr(&ctl->status, kStNonFinite);
        b = SINGLE ? 0 : g.atom_box[c];
        const int t = iperm[c];
        const double4_32a q = xb[t];
        const double qa[3] = {q.x, q.y, q.z};
        // a position equal to what md_get_state reports for the current
        // state (the current one wrapped into the box) keeps the current,
        // unwrapped representation: a state read back and loaded again is
        // the same state, bit for bit
        const double4_32a cur = x[t];
        const double ca[3] = {cur.x, cur.y, cur.z};
        double pa[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double L = g.L[3 * b + a];
            const double s = src[3 * c + a];
            if (wrap_step(ca[a], L) == s) {
                pa[a] = ca[a];
            } else {
                changed = true;
                const double w = wrap_coord(s, L);
                const double d = w - qa[a];
                pa[a] = d > 0.5 * L ? w - L : (d < -0.5 * L ? w + L : w);
            }
            const double e = pa[a] - qa[a];
            d2 = fma(e, e, d2);
        }
        if (changed) {
            const int ty = types[c];
            x[t] = make_double4_32a(pa[0], pa[1], pa[2], (double)ty);
            const double4_32a org = g.cell_org[cell_t[t]];
            xo[t] = make_float4((float)(pa[0] - org.x), (float)(pa[1] - org.y), (float)(pa[2] - org.z),
                                __int_as_float((int)__double_as_longlong(org.w) | (ty << 30)));
        }
    }
    if (__any_sync(0xffffffffu, changed) && (threadIdx.x & 31) == 0) atomicOr(&ctl->pos_changed, 1);
    record_disp<SINGLE>(g, N, b, d2, disp);
}

// After a state load that kept the lists: the displacement record restarts
// (each step recomputes it from the build positions) and the load's own
// list builds are not counted as builds of the dynamics.
__global__ void k_after_load(Ctl* ctl, int B, unsigned long long* __restrict__ disp) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) disp[b] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->n_rebuild = 0;
}

__global__ void k_load_vel(int64_t N, int64_t Np, const double* __restrict__ src, const int* __restrict__ iperm,
                           double* __restrict__ v, Ctl* ctl) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    if (src && (!isfinite(src[3 * c]) || !isfinite(src[3 * c + 1]) || !isfinite(src[3 * c + 2])))
        atomicOr(&ctl->status, kStNonFinite);
    int t = iperm[c];
    v[t] = src ? src[3 * c] : 0.0;
    v[Np + t] = src ? src[3 * c + 1] : 0.0;
    v[2 * Np + t] = src ? src[3 * c + 2] : 0.0;
}

__global__ void k_store_vec(int64_t N, int64_t Np, const double* __restrict__ soa, const double4_32a* __restrict__ x4,
                            const int* __restrict__ perm, double* __restrict__ dst, Geo g) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    int64_t c = perm[t];
    if (soa) {
        dst[3 * c] = soa[t];
        dst[3 * c + 1] = soa[Np + t];
        dst[3 * c + 2] = soa[2 * Np + t];
    } else {
        // positions leave the library wrapped into the box
        double4_32a p = x4[t];
        int b = g.B == 1 ? 0 : g.atom_box[t];
        dst[3 * c] = wrap_step(p.x, g.L[3 * b]);
        dst[3 * c + 1] = wrap_step(p.y, g.L[3 * b + 1]);
        dst[3 * c + 2] = wrap_step(p.z, g.L[3 * b + 2]);
    }
}

__global__ void k_store_scalar(int64_t N, const double* __restrict__ src, const int* __restrict__ perm,
                               double* __restrict__ dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    dst[perm[t]] = src[t];
}

__global__ void k_get_neighbors(int64_t N, int64_t Np, const int* __restrict__ nn, const int* __restrict__ nl,
                                int max_nb, const int* __restrict__ perm, int32_t* __restrict__ nn_out,
                                int32_t* __restrict__ nl_out, int32_t ld) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    int64_t c = perm[t];
    int n = nn[t];
    nn_out[c] = n;
    int m = min(min(n, max_nb), ld);
    for (int k = 0; k < m; ++k) nl_out[c * ld + k] = perm[entry_slot(nl[(int64_t)k * Np + t])];
}

__global__ void k_box_energy(int B, const double* __restrict__ thermo, double* __restrict__ e_box) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) e_box[b] = thermo[4 * b + 1];
}

__global__ void k_reset_perm(int64_t N, int* __restrict__ perm, int* __restrict__ iperm) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    perm[t] = (int)t;
    iperm[t] = (int)t;
}


void launch_load_positions(Engine& e, const double* src, cudaStream_t s) {
    if (e.N == 0) return;
    e.launches += 1;
    k_load_pos<<<nblk(e.N, 256), 256, 0, s>>>(e.N, src, e.iperm, make_geo(e), e.types, e.x, e.ctl);
}

void launch_load_positions_keep(Engine& e, const double* src, cudaStream_t s) {
    if (e.N == 0) return;
    e.launches += 1;
    if (single_fast(e))
        k_load_pos_keep<true><<<nblk(e.N, kINT), kINT, 0, s>>>(e.N, src, e.iperm, make_geo(e), e.x, e.xb, e.xo,
                                                             e.cell_t, e.types, e.ctl, e.disp_box);
    else
        k_load_pos_keep<false><<<nblk(e.N, kINT), kINT, 0, s>>>(e.N, src, e.iperm, make_geo(e), e.x, e.xb, e.xo,
                                                              e.cell_t, e.types, e.ctl, e.disp_box);
}

// New species for the current state: positions' pad lanes and the type
// bits of the float32 offsets, in sorted order.
__global__ void k_apply_types(int64_t N, const int* __restrict__ perm, const int* __restrict__ types,
                              double4_32a* __restrict__ x, float4* __restrict__ xo) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const int ty = types[perm[t]];
        x[t].w = (double)ty;
        float4 o = xo[t];
        o.w = __int_as_float((__float_as_int(o.w) & 0x3fffffff) | (ty << 30));
        xo[t] = o;
    }
}

void launch_apply_types(Engine& e, cudaStream_t s) {
    if (e.N == 0) return;
    e.launches += 1;
    k_apply_types<<<(int)std::min<int64_t>(nblk(e.N, 256), (int64_t)8 * e.n_sm), 256, 0, s>>>(e.N, e.perm, e.types,
                                                                                               e.x, e.xo);
}

void launch_after_load(Engine& e, cudaStream_t s) {
    e.launches += 1;
    k_after_load<<<std::max(1, std::min((e.B + 255) / 256, 64)), 256, 0, s>>>(e.ctl, e.B, e.disp_box);
}

void launch_load_velocities(Engine& e, const double* src, cudaStream_t s) {
    if (e.N == 0) return;
    e.launches += 1;
    k_load_vel<<<nblk(e.N, 256), 256, 0, s>>>(e.N, e.N_pad, src, e.iperm, e.v, e.ctl);
}

void launch_store_vec(Engine& e, const double* soa, const double4_32a* x4, double* dst, cudaStream_t s) {
    if (e.N == 0) return;
    e.launches += 1;
    k_store_vec<<<nblk(e.N, 256), 256, 0, s>>>(e.N, e.N_pad, soa, x4, e.perm, dst, make_geo(e));
}

void launch_store_scalar(Engine& e, const double* src, double* dst, cudaStream_t s) {
    if (e.N == 0) return;
    e.launches += 1;
    k_store_scalar<<<nblk(e.N, 256), 256, 0, s>>>(e.N, src, e.perm, dst);
}

void launch_get_neighbors(Engine& e, int32_t* nn_out, int32_t* nl_out, int32_t ld, cudaStream_t s) {
    if (e.N == 0) return;
    e.launches += 1;
    k_get_neighbors<<<nblk(e.N, 256), 256, 0, s>>>(e.N, e.N_pad, e.nn, e.nl, e.max_nb, e.perm, nn_out, nl_out, ld);
}

void launch_box_energy(Engine& e, double* e_box, cudaStream_t s) {
    e.launches += 1;
    k_box_energy<<<nblk(e.B, 256), 256, 0, s>>>(e.B, e.thermo_dev, e_box);
}

void launch_reset_perm(Engine& e, cudaStream_t s) {
    if (e.N == 0) return;
    e.launches += 1;
    k_reset_perm<<<nblk(e.N, 256), 256, 0, s>>>(e.N, e.perm, e.iperm);
}

// ---------------------------------------------------------------- diagnostics

__global__ void k_eval_math(int fn, const double* __restrict__ x, int64_t n, double* __restrict__ out,
                            const double* __restrict__ gT, ExpConst K) {
    __shared__ double sT[kExpTable];
    load_exp_table(sT, gT);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = x[i];
    switch (fn) {
        case 0: out[i] = exp_tab(v, sT, K); break;
        case 1: out[i] = exp(v); break;
        case 2: out[i] = rsqrt_nr(v); break;
        case 3: out[i] = rsqrt(v); break;
        default: {
            double y, r;
            rsqrt_sqrt(v, y, r);
            out[i] = fn == 4 ? y : r;
        }
    }
}

void launch_eval_math(Engine& e, int fn, const double* x, int64_t n, double* out, cudaStream_t s) {
    if (n <= 0) return;
    e.launches += 1;
    k_eval_math<<<nblk(n, 256), 256, 0, s>>>(fn, x, n, out, e.exp_T, e.exp_const);
}

// ---------------------------------------------------------------- splines

// Natural cubic spline through knot values y_0..y_{n-1} on a uniform grid of
// spacing h: second derivatives M from the tridiagonal system
//   (h/6) M_{k-1} + (2h/3) M_k + (h/6) M_{k+1} = (y_{k+1} - 2 y_k + y_{k-1}) / h,
// M_0 = M_{n-1} = 0 (Thomas algorithm), then per-interval coefficients of
//   s(u) = y_k + b u + c u^2 + d u^3, u = t - t_k,
//   b = (y_{k+1} - y_k)/h - h (2 M_k + M_{k+1})/6, c = M_k/2, d = (M_{k+1} - M_k)/(6h);
// entry n-1 holds the value and slope at the last knot (extrapolation).
// One thread per spline table: np_ V tables (n0 knots), np_ rho tables (n1)
// and nt F tables (n2), back to back as the knot values are.
__global__ void k_spline_setup(const double* __restrict__ y_all, double* __restrict__ work,
                               double4_32a* __restrict__ coef, float4* __restrict__ coef_f, int n0, int n1, int n2,
                               double h0, double h1, double h2, int np_, int nt) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= 2 * np_ + nt) return;
    const int kind = w < np_ ? 0 : (w < 2 * np_ ? 1 : 2);
    const int n = kind == 0 ? n0 : (kind == 1 ? n1 : n2);
    const int off = kind == 0 ? w * n0 : (kind == 1 ? np_ * n0 + (w - np_) * n1 : np_ * (n0 + n1) + (w - 2 * np_) * n2);
    const double h = kind == 0 ? h0 : (kind == 1 ? h1 : h2);
    const double* y = y_all + off;
    double* cp = work + 3 * off;  // modified super-diagonal
    double* dp = cp + n;          // modified right-hand side
    double* M = dp + n;
    double a = h / 6.0, bd = 2.0 * h / 3.0, cu = h / 6.0;
    for (int k = 1; k <= n - 2; ++k) {
        double rhs = (y[k + 1] - 2.0 * y[k] + y[k - 1]) / h;
        double den = k == 1 ? bd : bd - a * cp[k - 1];
        cp[k] = cu / den;
        dp[k] = (k == 1 ? rhs : rhs - a * dp[k - 1]) / den;
    }
    M[0] = 0.0;
    M[n - 1] = 0.0;
    for (int k = n - 2; k >= 1; --k) M[k] = dp[k] - (k < n - 2 ? cp[k] * M[k + 1] : 0.0);
    double4_32a* c = coef + off;
    for (int k = 0; k < n - 1; ++k) {
        double b = (y[k + 1] - y[k]) / h - h * (2.0 * M[k] + M[k + 1]) / 6.0;
        c[k] = make_double4_32a(y[k], b, 0.5 * M[k], (M[k + 1] - M[k]) / (6.0 * h));
    }
    double4_32a l = c[n - 2];
    c[n - 1] = make_double4_32a(y[n - 1], l.y + 2.0 * l.z * h + 3.0 * l.w * h * h, 0.0, 0.0);
    float4* cf = coef_f + off;
    for (int k = 0; k < n; ++k) cf[k] = make_float4((float)c[k].x, (float)c[k].y, (float)c[k].z, (float)c[k].w);
}

// Float64 pair records from the V and rho coefficients of each type pair
// (both on the grid t_k = r_lo + k h, n knots): record 0 continues interval
// 0 linearly below r_lo, record k + 1 is interval k, record n continues
// linearly above r_hi with the end value and slope. Derivative coefficients
// 2 c2 and 3 c3 are stored beside c0..c3.
__global__ void k_pair_records(const double4_32a* __restrict__ coef, double4_32a* __restrict__ rec, int n,
                               double t0, double h, int np_) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np_ * (n + 1)) return;
    const int pt = t / (n + 1), q = t % (n + 1);
    const double4_32a* cv = coef + (int64_t)pt * n;             // V of pair pt
    const double4_32a* cr = coef + (int64_t)np_ * n + (int64_t)pt * n;  // rho of pair pt
    double tk;
    double4_32a v, f;
    if (q == 0) {
        tk = t0;
        v = make_double4_32a(cv[0].x, cv[0].y, 0.0, 0.0);
        f = make_double4_32a(cr[0].x, cr[0].y, 0.0, 0.0);
    } else if (q == n) {
        tk = fma(h, (double)(n - 1), t0);
        v = make_double4_32a(cv[n - 1].x, cv[n - 1].y, 0.0, 0.0);
        f = make_double4_32a(cr[n - 1].x, cr[n - 1].y, 0.0, 0.0);
    } else {
        tk = fma(h, (double)(q - 1), t0);
        v = cv[q - 1];
        f = cr[q - 1];
    }
    double4_32a* o = rec + (int64_t)t * 4;
    o[0] = make_double4_32a(tk, v.x, v.y, v.z);
    o[1] = make_double4_32a(v.w, 2.0 * v.z, 3.0 * v.w, f.x);
    o[2] = make_double4_32a(f.y, f.z, f.w, 2.0 * f.z);
    o[3] = make_double4_32a(3.0 * f.w, 0.0, 0.0, 0.0);
}

void launch_spline_setup(Engine& e, cudaStream_t s) {
    const md_potential& p = e.pot_host;
    e.launches += 1;
    const int nt = std::max(p.n_types, 1), np_ = nt * (nt + 1) / 2;
    k_spline_setup<<<(2 * np_ + nt + 31) / 32, 32, 0, s>>>(e.knots_dev, e.spline_work, e.spline_coef,
                                                            e.spline_coef_f, p.n_phi, p.n_f, p.n_F, e.pot.sh[0],
                                                            e.pot.sh[1], e.pot.sh[2], np_, nt);
    if (e.spline_pair_rec) {
        e.launches += 1;
        const int nrec = np_ * (p.n_phi + 1);
        k_pair_records<<<(nrec + 127) / 128, 128, 0, s>>>(e.spline_coef, e.spline_pair_rec, p.n_phi, e.pot.st0[0],
                                                          e.pot.sh[0], np_);
    }
}

}  // namespace mdk
