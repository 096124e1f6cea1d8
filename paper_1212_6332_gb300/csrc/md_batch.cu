// Block-per-box schedule for batches of small boxes (Sec. 4.4).
//
// The paper combines many small boxes into one large run so that one launch
// covers all of them. The tile schedule (the regular kernels over the
// atoms of all boxes) does that phase by phase. This schedule goes further:
// one thread block owns one box for all n_steps steps and keeps its
// positions and F'(rho) in shared memory (a 4000-atom box needs 192 KB of
// the 227 KB a block may hold), so a step needs no launch, no grid-wide
// synchronization and no global gather of neighbour positions. Each box
// decides its own list rebuild and re-sorts its own atoms inside the block:
//   kick-drift -> [wrap, bin, counting sort, list build] -> density -> force
// with __syncthreads between phases; the pair functions are evaluated once
// per pair (from the lower slot, both cache slots written through the
// reverse index) and summed in list order, the arithmetic and the order of
// the tile kernels, so both schedules give the same bits.
// Boxes are launched largest first in shared-memory size classes.
#include <algorithm>
#include <vector>

#include "md_device.cuh"

namespace mdk {

struct BoxArgs {
    int64_t Np;
    int max_nb;
    double rl2;
    float rl2f_lo, rl2f_hi;
    double c_kick, dt, half_skin2;
    Bath bath;
    double4_32a* x;
    double4_32a* x_alt;
    double4_32a* xb;
    double* v;
    double* v_alt;
    double* f;
    double* rho;
    double* Fp;
    double* e_atom;
    float4* xo;
    int* perm;
    int* perm_alt;
    int* iperm;
    int* cell_t;
    int* nn;
    int* nl;
    double2* ab;  // (V'/r, rho'/r) halves of the float64 pair cache entries: ab[2 slot]
    double4_32a* pc;  // the whole 32-byte entries (V'/r, rho'/r, rho, V)
    int* n_up;  // float64 tile path's list layout data, kept valid across schedules
    int* rev;
    int* nl_lo;  // row-major lower parts for the reverse-index search
    int sum_S;  // word split of the fixed-point density sums (sum_split)
    int cut_bits;  // 2^cut_bits > r_cut, for the force sums' separation split (DSplit)
    Ctl* ctl;
    int* box_done;
    int* box_state;
    const int* box_order;
};

// Rebuild inside the block: wrap, bin, sort by caller id within each cell,
// permute, list build. Returns the largest list length of the box.
__device__ int box_rebuild(const Geo& g, const BoxArgs& A, int b, int64_t a0, int nb, int c0, int ncl,
                           double4_32a* sx, int* s_ord, int* s_cell, int* s_cnt, int* s_start, int* s_max) {
    const int tid = threadIdx.x, NT = blockDim.x;
    const double L[3] = {g.L[3 * b], g.L[3 * b + 1], g.L[3 * b + 2]};
    const int nc[3] = {g.nc[3 * b], g.nc[3 * b + 1], g.nc[3 * b + 2]};
    for (int c = tid; c <= ncl; c += NT) s_cnt[c] = 0;
    if (tid == 0) *s_max = 0;
    __syncthreads();
    for (int t = tid; t < nb; t += NT) {
        double4_32a p = sx[t];
        p.x = wrap_step(p.x, L[0]);
        p.y = wrap_step(p.y, L[1]);
        p.z = wrap_step(p.z, L[2]);
        sx[t] = p;
        double pc[3] = {p.x, p.y, p.z};
        int cc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int k = (int)floor(pc[a] / g.cell_len[3 * b + a]);
            cc[a] = k < 0 ? 0 : (k >= nc[a] ? nc[a] - 1 : k);
        }
        int local = g.cell_rank[c0 + (cc[0] * nc[1] + cc[1]) * nc[2] + cc[2]] - c0;
        s_cell[t] = local;
        atomicAdd(&s_cnt[local], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int c = 0; c < ncl; ++c) {
            s_start[c] = run;
            run += s_cnt[c];
            s_cnt[c] = 0;
        }
        s_start[ncl] = run;
    }
    __syncthreads();
    for (int t = tid; t < nb; t += NT) {
        int c = s_cell[t];
        s_ord[s_start[c] + atomicAdd(&s_cnt[c], 1)] = t;
    }
    __syncthreads();
    // order each cell by caller id; record the cell of every new slot
    for (int c = tid; c < ncl; c += NT) {
        int lo = s_start[c], hi = s_start[c + 1];
        for (int k = lo + 1; k < hi; ++k) {
            int s = s_ord[k];
            int key = A.perm[a0 + s];
            int j = k - 1;
            while (j >= lo && A.perm[a0 + s_ord[j]] > key) {
                s_ord[j + 1] = s_ord[j];
                --j;
            }
            s_ord[j + 1] = s;
        }
        for (int k = lo; k < hi; ++k) s_cell[k] = c;
    }
    // stage the old order in the alternate global buffers
    for (int t = tid; t < nb; t += NT) {
        A.x_alt[a0 + t] = sx[t];
        A.v_alt[a0 + t] = A.v[a0 + t];
        A.v_alt[A.Np + a0 + t] = A.v[A.Np + a0 + t];
        A.v_alt[2 * A.Np + a0 + t] = A.v[2 * A.Np + a0 + t];
        A.perm_alt[a0 + t] = A.perm[a0 + t];
    }
    __syncthreads();
    for (int k = tid; k < nb; k += NT) {
        int s = s_ord[k];
        double4_32a p = A.x_alt[a0 + s];
        sx[k] = p;
        A.xb[a0 + k] = p;
        A.v[a0 + k] = A.v_alt[a0 + s];
        A.v[A.Np + a0 + k] = A.v_alt[A.Np + a0 + s];
        A.v[2 * A.Np + a0 + k] = A.v_alt[2 * A.Np + a0 + s];
        int id = A.perm_alt[a0 + s];
        A.perm[a0 + k] = id;
        A.iperm[id] = (int)(a0 + k);
        int gc = c0 + s_cell[k];
        A.cell_t[a0 + k] = gc;
        A.xo[a0 + k] = cell_local(g, b, gc, p);
    }
    __syncthreads();
    // list build: a warp per centre atom, candidates of the (de-duplicated)
    // 27-cell stencil in the tile kernel's order, 32 per lane step
    const int lane = tid & 31, warp = tid >> 5, nw = NT >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const float lf[3] = {g.cell_len_f[3 * b], g.cell_len_f[3 * b + 1], g.cell_len_f[3 * b + 2]};
    const float Lf[3] = {(float)L[0], (float)L[1], (float)L[2]};
    int my_max = 0;
    for (int i = warp; i < nb; i += nw) {
        const float4 oi = A.xo[a0 + i];
        const double4_32a xi = sx[i];
        const int ci = __float_as_int(oi.w);
        const int cix = ci & 1023, ciy = (ci >> 10) & 1023, ciz = (ci >> 20) & 1023;
        int qs[27];
        const int n_st = stencil_sorted(g, b, cix, ciy, ciz, qs);
        int n = 0;
        for (int st = 0; st < n_st; ++st) {
                    int q = qs[st] - c0;
                    int lo = s_start[q], hi = s_start[q + 1];
                    for (int jb = lo; jb < hi; jb += 32) {
                        int jj = jb + lane;
                        bool ok = false;
                        int sxv = 0, syv = 0, szv = 0;
                        if (jj < hi) {
                            ok = list_candidate(oi, A.xo[a0 + jj], xi, sx, jj, cix, ciy, ciz, nc[0], nc[1], nc[2],
                                                lf[0], lf[1], lf[2], Lf[0], Lf[1], Lf[2], L[0], L[1], L[2], A.rl2,
                                                A.rl2f_lo, A.rl2f_hi, sxv, syv, szv) &&
                                 (jj != i);
                        }
                        unsigned m = __ballot_sync(0xffffffffu, ok);
                        if (ok) {
                            int pos = n + __popc(m & lt_mask);
                            if (pos < A.max_nb)
                                A.nl[(int64_t)pos * A.Np + a0 + i] = make_entry((int)(a0 + jj), sxv, syv, szv);
                        }
                        n += __popc(m);
                    }
        }
        if (lane == 0) A.nn[a0 + i] = n;
        my_max = max(my_max, n);
    }
    if (lane == 0) atomicMax(s_max, my_max);
    __syncthreads();
    // the same [upper | lower] layout and reverse index as the tile path,
    // so either schedule can continue from the other
    if (*s_max <= A.max_nb) {
        for (int t = tid; t < nb; t += NT)
            A.n_up[a0 + t] = rotate_list(A.Np, a0 + t, min(A.nn[a0 + t], A.max_nb), A.nl, A.nl_lo, A.max_nb);
        __syncthreads();
        for (int t = tid; t < nb; t += NT)
            reverse_index(A.Np, a0 + t, min(A.nn[a0 + t], A.max_nb), A.n_up[a0 + t], A.nn, A.nl, A.nl_lo, A.n_up,
                          A.max_nb, A.rev);
        __syncthreads();
    }
    return *s_max;
}

template <int KIND>
__global__ void k_box_steps(Geo g, Pot P, BoxArgs A, int n_steps) {
    extern __shared__ double4_32a smem_box[];
    __shared__ double sT[kExpTable];
    __shared__ double s_red[32];
    __shared__ int s_flag, s_max;
    const int b = A.box_order[blockIdx.x];
    const int64_t a0 = g.atom_off[b];
    const int nb = (int)(g.atom_off[b + 1] - a0);
    const int c0 = g.cell_off[b], ncl = g.cell_off[b + 1] - c0;
    const int tid = threadIdx.x, NT = blockDim.x;
    double4_32a* sx = smem_box;
    double* sFp = (double*)(sx + nb);
    int* s_ord = (int*)(sFp + nb);
    int* s_cell = s_ord + nb;
    int* s_cnt = s_cell + nb;
    int* s_start = s_cnt + ncl + 1;
    if (KIND == MD_POT_RGL) load_exp_table(sT, P.exp_T);
    if (nb == 0) return;
    const double L[3] = {g.L[3 * b], g.L[3 * b + 1], g.L[3 * b + 2]};
    const int kq = box_kq(L[0], L[1], L[2]);
    const long long qL[3] = {to_fixed(L[0], kq), to_fixed(L[1], kq), to_fixed(L[2], kq)};
    for (int t = tid; t < nb; t += NT) sx[t] = A.x[a0 + t];
    int done = A.box_done[b];
    bool pending = A.box_state[b] == 1;
    __syncthreads();
    while (done < n_steps) {
        bool rebuild = pending;
        if (!pending) {
            double m = 0.0;
            for (int t = tid; t < nb; t += NT) {
                const int64_t i = a0 + t;
                double4_32a p = sx[t];
                double4_32a q = A.xb[i];
                double vx = A.v[i], vy = A.v[A.Np + i], vz = A.v[2 * A.Np + i];
                bath_half(A.bath, vx, vy, vz);  // friction half step before the kick
                vx = vx + A.c_kick * A.f[i];
                vy = vy + A.c_kick * A.f[A.Np + i];
                vz = vz + A.c_kick * A.f[2 * A.Np + i];
                p.x += A.dt * vx;
                p.y += A.dt * vy;
                p.z += A.dt * vz;
                A.v[i] = vx;
                A.v[A.Np + i] = vy;
                A.v[2 * A.Np + i] = vz;
                sx[t] = p;
                double dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
                double d2 = dx * dx + dy * dy + dz * dz;
                m = d2 > m ? d2 : m;
            }
            m = warp_max(m);
            if ((tid & 31) == 0) s_red[tid >> 5] = m;
            __syncthreads();
            if (tid == 0) {
                double mm = 0.0;
                for (int k = 0; k < (NT >> 5); ++k) mm = s_red[k] > mm ? s_red[k] : mm;
                s_flag = mm > A.half_skin2;
            }
            __syncthreads();
            rebuild = s_flag != 0;
        }
        pending = false;
        if (rebuild) {
            int mx = box_rebuild(g, A, b, a0, nb, c0, ncl, sx, s_ord, s_cell, s_cnt, s_start, &s_max);
            if (tid == 0) {
                atomicAdd((unsigned long long*)&A.ctl->n_rebuild, 1ULL);
                atomicMax(&A.ctl->max_count, mx);
            }
            if (mx > A.max_nb) {
                // the drift of this step is done and the atoms are sorted;
                // the host grows the list and relaunches from here
                if (tid == 0) {
                    A.box_state[b] = 1;
                    A.box_done[b] = done;
                    atomicOr(&A.ctl->status, kStOverflow);
                    atomicMax(&A.ctl->overflow_count, mx);
                }
                for (int t = tid; t < nb; t += NT) A.x[a0 + t] = sx[t];
                return;
            }
        }
        // pair functions once per pair, as the tile schedule's pair pass:
        // the atom of the lower slot evaluates each of its upper entries
        // (j > i) and writes the 32-byte entry to its slot and, through the
        // reverse index, to the partner's
        for (int t = tid; t < nb; t += NT) {
            const int64_t i = a0 + t;
            const double4_32a xi = sx[t];
            const long long qi[3] = {to_fixed(xi.x, kq), to_fixed(xi.y, kq), to_fixed(xi.z, kq)};
            const int nup = A.n_up[i];
            const int n = nup < 0 ? min(A.nn[i], A.max_nb) : nup;
            for (int k = 0; k < n; ++k) {
                const int64_t slot = (int64_t)k * A.Np + i;
                const int e = A.nl[slot];
                const int jg = entry_slot(e);
                if (jg <= i) continue;
                const double r2 = r2_exact(qi, sx[jg - a0], entry_code(e), qL, kq);
                double Av = 0.0, Bv = 0.0, phi = 0.0, fr = 0.0;
                if (below(r2, P.rc2)) pair_eval<KIND>(P, sT, r2, phi, fr, Av, Bv);
                const double4_32a c = make_double4_32a(Av, Bv, fr, phi);
                A.pc[slot] = c;
                A.pc[(int64_t)A.rev[slot] * A.Np + jg] = c;
            }
        }
        __syncthreads();
        // density sums: the fixed-point totals of the cached values, which
        // the tile schedule's pair pass forms by atomic adds of the same
        // terms (integer sums: the same bits in any order)
        for (int t = tid; t < nb; t += NT) {
            const int64_t i = a0 + t;
            const int n = min(A.nn[i], A.max_nb);
            FixedSum qr, qv;
            bool ok = true;
            for (int k = 0; k < n; ++k) {
                const double2 w = cache_fv(A.pc, (int64_t)k * A.Np + i);
                ok &= qr.add(w.x, A.sum_S) & qv.add(w.y, A.sum_S);
            }
            if (!ok) atomicOr(&A.ctl->status, kStNonFinite);
            double r_i, Fpi, E;
            embed_sums<KIND>(P, qr, qv, A.sum_S, 0, A.pc, A.Np, i, n, r_i, Fpi, E);
            A.rho[i] = r_i;
            A.Fp[i] = Fpi;
            sFp[t] = Fpi;
            A.e_atom[i] = E;
        }
        __syncthreads();
        // force pass and second half-kick
        for (int t = tid; t < nb; t += NT) {
            const int64_t i = a0 + t;
            const double4_32a xi = sx[t];
            const double Fpi = sFp[t];
            const int n = min(A.nn[i], A.max_nb);
            // the tile schedule's sum of s_ij (x_j - x_i), the separation in
            // its fixed point, in float32 pieces in the same order: the same bits
            const DSplit D = dsplit_init(kq, A.cut_bits);
            const long long qi[3] = {to_fixed(xi.x, kq) - D.rnd, to_fixed(xi.y, kq) - D.rnd,
                                     to_fixed(xi.z, kq) - D.rnd};
            ForceSumF fs;
            for (int k = 0; k < n; ++k) {
                const int64_t slot = (int64_t)k * A.Np + i;
                double2 c = A.ab[2 * slot];
                if ((__double_as_longlong(c.x) | __double_as_longlong(c.y)) == 0) continue;
                const int e = A.nl[slot];
                const int jl = entry_slot(e) - (int)a0;
                const unsigned code = entry_code(e);
                const double4_32a xj = sx[jl];
                const double s = fma(Fpi + sFp[jl], c.y, c.x);
                long long rx = to_fixed(xj.x, kq) - qi[0], ry = to_fixed(xj.y, kq) - qi[1],
                          rz = to_fixed(xj.z, kq) - qi[2];
                if (code != kNoShift) {
                    rx += qshift(code, 0, qL[0]);
                    ry += qshift(code, 1, qL[1]);
                    rz += qshift(code, 2, qL[2]);
                }
                fs.add(s, rx, ry, rz, D);
            }
            const double fx = fs.value(0), fy = fs.value(1), fz = fs.value(2);
            A.f[i] = fx;
            A.f[A.Np + i] = fy;
            A.f[2 * A.Np + i] = fz;
            double vx = A.v[i] + A.c_kick * fx, vy = A.v[A.Np + i] + A.c_kick * fy;
            double vz = A.v[2 * A.Np + i] + A.c_kick * fz;
            bath_half(A.bath, vx, vy, vz);  // friction half step after the kick
            A.v[i] = vx;
            A.v[A.Np + i] = vy;
            A.v[2 * A.Np + i] = vz;
        }
        __syncthreads();
        ++done;
    }
    for (int t = tid; t < nb; t += NT) A.x[a0 + t] = sx[t];
    if (tid == 0) {
        A.box_done[b] = done;
        A.box_state[b] = 0;
    }
}

static size_t box_smem(int atoms, int cells) {
    return (size_t)atoms * (32 + 8 + 4 + 4) + (size_t)(cells + 1) * 8;
}

constexpr size_t kBoxSmemMax = 200 * 1024;

bool box_schedule_fits(const Engine& e) {
    // float64 and one species only; the pressure coupling scales boxes
    // between steps, which the in-block step loop does not do
    if (e.cfg.precision != MD_FP64 || e.baro.on || e.pot.n_types > 1) return false;
    for (int b = 0; b < e.B; ++b) {
        int nb = (int)(e.atom_off_h[b + 1] - e.atom_off_h[b]);
        int ncl = e.cell_off_h[b + 1] - e.cell_off_h[b];
        if (box_smem(nb, ncl) > kBoxSmemMax) return false;
    }
    return true;
}

// Groups boxes into shared-memory classes (largest first inside a class)
// and uploads the launch order.
static int box_setup(Engine& e) {
    if (e.box_order) return MD_OK;
    std::vector<int> idx(e.B);
    for (int b = 0; b < e.B; ++b) idx[b] = b;
    auto atoms = [&](int b) { return (int)(e.atom_off_h[b + 1] - e.atom_off_h[b]); };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return atoms(a) > atoms(c); });
    const int caps[4] = {4608, 2048, 1024, 512};
    e.box_classes.clear();
    size_t k = 0;
    for (int ci = 0; ci < 4 && k < idx.size(); ++ci) {
        int cap = caps[ci];
        int next_cap = ci + 1 < 4 ? caps[ci + 1] : 0;
        BoxClass c{};
        c.first = (int)k;
        int max_cells = 0, max_atoms = 0;
        while (k < idx.size() && atoms(idx[k]) > next_cap && atoms(idx[k]) <= cap) {
            max_atoms = std::max(max_atoms, atoms(idx[k]));
            max_cells = std::max(max_cells, e.cell_off_h[idx[k] + 1] - e.cell_off_h[idx[k]]);
            ++k;
        }
        c.count = (int)k - c.first;
        if (c.count == 0) continue;
        c.smem = box_smem(max_atoms, max_cells);
        c.threads = max_atoms > 1024 ? 512 : (max_atoms > 256 ? 256 : 128);
        e.box_classes.push_back(c);
    }
    if (k != idx.size()) return MD_ERR_UNSUPPORTED;
    if (cudaMalloc(&e.box_order, sizeof(int) * e.B) != cudaSuccess ||
        cudaMalloc(&e.box_done, sizeof(int) * e.B) != cudaSuccess ||
        cudaMalloc(&e.box_state, sizeof(int) * e.B) != cudaSuccess) {
        cudaGetLastError();
        return MD_ERR_NOMEM;
    }
    if (cudaMemcpy(e.box_order, idx.data(), sizeof(int) * e.B, cudaMemcpyHostToDevice) != cudaSuccess)
        return MD_ERR_CUDA;
    return MD_OK;
}

template <int KIND>
static void box_launch(Engine& e, int n_steps, cudaStream_t s) {
    Geo g = make_geo(e);
    BoxArgs A{};
    A.Np = e.N_pad;
    A.max_nb = e.max_nb;
    A.rl2 = e.rl * e.rl;
    double margin = 4e-4 * e.rl;
    A.rl2f_lo = (float)(A.rl2 - margin);
    A.rl2f_hi = (float)(A.rl2 + margin);
    A.c_kick = 0.5 * e.cfg.dt / (e.cfg.mass * kMVV);
    A.bath = e.bath;
    A.dt = e.cfg.dt;
    A.half_skin2 = 0.25 * e.cfg.skin * e.cfg.skin;
    A.x = e.x;
    A.x_alt = e.x_alt;
    A.xb = e.xb;
    A.v = e.v;
    A.v_alt = e.v_alt;
    A.f = e.f;
    A.rho = e.rho;
    A.Fp = e.Fp;
    A.e_atom = e.e_atom;
    A.xo = e.xo;
    A.perm = e.perm;
    A.perm_alt = e.perm_alt;
    A.iperm = e.iperm;
    A.cell_t = e.cell_t;
    A.nn = e.nn;
    A.nl = e.nl;
    A.ab = reinterpret_cast<double2*>(e.pc);
    A.pc = e.pc;
    A.n_up = e.n_up;
    A.rev = e.rev;
    A.nl_lo = e.nl_lo;
    A.sum_S = sum_split(e.max_nb);
    A.cut_bits = cut_bits(e.pot.rc);
    A.ctl = e.ctl;
    A.box_done = e.box_done;
    A.box_state = e.box_state;
    for (const BoxClass& c : e.box_classes) {
        A.box_order = e.box_order + c.first;
        if (c.smem > 48 * 1024)
            cudaFuncSetAttribute(k_box_steps<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
        k_box_steps<KIND><<<c.count, c.threads, c.smem, s>>>(g, e.pot, A, n_steps);
        e.launches += 1;
    }
}

int launch_box_steps(Engine& e, int n_steps, bool first, cudaStream_t s) {
    if (e.N == 0 || n_steps == 0) return MD_OK;
    int rc = box_setup(e);
    if (rc) return rc;
    if (first) {
        if (cudaMemsetAsync(e.box_done, 0, sizeof(int) * e.B, s) != cudaSuccess ||
            cudaMemsetAsync(e.box_state, 0, sizeof(int) * e.B, s) != cudaSuccess)
            return MD_ERR_CUDA;
    }
    PhaseScope scope(e, MD_PHASE_FORCE, s);
    switch (e.pot.kind) {
        case MD_POT_RGL: box_launch<MD_POT_RGL>(e, n_steps, s); break;
        case MD_POT_SC: box_launch<MD_POT_SC>(e, n_steps, s); break;
        default: box_launch<MD_POT_SPLINE>(e, n_steps, s); break;
    }
    return cudaGetLastError() == cudaSuccess ? MD_OK : MD_ERR_CUDA;
}

}  // namespace mdk
