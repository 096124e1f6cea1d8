// Cell binning and sorting (Sec. 3.2, Fig. 2): the paper computes each
// atom's cell on the GPU and builds linked lists and the sorted order on the
// host. Here the whole partition runs on the device as a counting sort:
//   k_bin          cell of every atom, atomic count per cell
//   k_scan_*       exclusive scan of the counts -> first atom of each cell
//   k_scatter      atomic slot inside the cell
//   k_sort_cells   order each cell's atoms by caller id (deterministic)
//   k_permute      gather x, v, ids into the new order (alternate buffers)
//   k_copy_back    copy back, record positions at build, inverse map
// Every box decides on the device whether it rebuilds (mode 1, or its
// largest displacement since its last build exceeds skin/2); atoms and cells
// of the other boxes are left untouched, so the chain can be launched every
// step, or captured in a CUDA graph, without a host decision.
#include <algorithm>
#include <cstring>

#include "md_device.cuh"

namespace mdk {

// The per-atom kernels below loop over the atoms with a fixed grid (a few
// waves of resident blocks) and read the status word once, so a step that
// rebuilds nothing costs a few microseconds per kernel.

__global__ void k_bin(int64_t N, double4_32a* __restrict__ x, Geo g, int* __restrict__ cell_of,
                      int* __restrict__ cell_count, const Ctl* ctl, const unsigned long long* __restrict__ disp,
                      int mode, unsigned long long thr) {
    if (load_status(ctl)) return;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        int b = g.B == 1 ? 0 : g.atom_box[s];
        if (!box_due(disp, b, mode, thr)) continue;
        // positions drift unwrapped between builds; wrap them into the box here
        double4_32a p = x[s];
        p.x = wrap_step(p.x, g.L[3 * b]);
        p.y = wrap_step(p.y, g.L[3 * b + 1]);
        p.z = wrap_step(p.z, g.L[3 * b + 2]);
        x[s] = p;
        double pc[3] = {p.x, p.y, p.z};
        int c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int n = g.nc[3 * b + a];
            int k = (int)floor(pc[a] / g.cell_len[3 * b + a]);
            c[a] = k < 0 ? 0 : (k >= n ? n - 1 : k);
        }
        int lin = g.cell_off[b] + (c[0] * g.nc[3 * b + 1] + c[1]) * g.nc[3 * b + 2] + c[2];
        int gc = g.cell_rank[lin];
        cell_of[s] = gc;
        atomicAdd(&cell_count[gc], 1);
    }
}

constexpr int kScanNT = 1024;

// Exclusive scan of counts[0..n) within blocks of kScanNT; block totals out.
__global__ void k_scan_blocks(int n, const int* __restrict__ counts, int* __restrict__ start,
                              int* __restrict__ block_tot, const Ctl* ctl) {
    if (load_status(ctl)) return;
    __shared__ int wsum[kScanNT / 32];
    int i = blockIdx.x * kScanNT + threadIdx.x;
    int v = i < n ? counts[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int s = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        wsum[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    int excl = incl - v + (w > 0 ? wsum[w - 1] : 0);
    if (i < n) start[i] = excl;
    if (threadIdx.x == kScanNT - 1) block_tot[blockIdx.x] = wsum[31];
}

// One block: exclusive scan of the block totals, serially over chunks.
__global__ void k_scan_totals(int nb, int* __restrict__ block_tot, const Ctl* ctl) {
    if (load_status(ctl)) return;
    __shared__ int wsum[kScanNT / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += kScanNT) {
        int i = base + threadIdx.x;
        int v = i < nb ? block_tot[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            int s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        int excl = incl - v + (w > 0 ? wsum[w - 1] : 0) + carry;
        if (i < nb) block_tot[i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
}

// Adds block offsets, zeroes the counts (they become fill counters) and
// closes the prefix array. The result S is an exclusive prefix over the
// counted atoms of all cells; the atoms of cell c of box b occupy
// [atom_off[b] + S[c] - S[cell_off[b]], atom_off[b] + S[c+1] - S[cell_off[b]])
// (cell_range), so boxes that keep their lists are left where they are.
__global__ void k_scan_add(int n, int* __restrict__ start, const int* __restrict__ block_tot,
                           int* __restrict__ counts, const Ctl* ctl) {
    if (load_status(ctl)) return;
    int i = blockIdx.x * kScanNT + threadIdx.x;
    if (i < n) {
        int v = counts[i];
        start[i] += block_tot[blockIdx.x];
        counts[i] = 0;
        if (i == n - 1) start[n] = start[i] + v;
    }
}

__global__ void k_scatter(int64_t N, Geo g, const int* __restrict__ cell_of, const int* __restrict__ start,
                          int* __restrict__ fill, int* __restrict__ src, const Ctl* ctl,
                          const unsigned long long* __restrict__ disp, int mode, unsigned long long thr) {
    if (load_status(ctl)) return;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        int b = g.B == 1 ? 0 : g.atom_box[s];
        if (!box_due(disp, b, mode, thr)) continue;
        int c = cell_of[s];
        int64_t t = g.atom_off[b] + (start[c] - start[g.cell_off[b]]) + atomicAdd(&fill[c], 1);
        src[t] = (int)s;
    }
}

// Orders the atoms of each cell by caller id, so the sorted order (and every
// sum over it) does not depend on the atomic order of k_scatter.
__global__ void k_sort_cells(int n_cells, Geo g, const int* __restrict__ start, int* __restrict__ fill,
                             int* __restrict__ src, const int* __restrict__ perm, const Ctl* ctl,
                             const unsigned long long* __restrict__ disp, int mode, unsigned long long thr) {
    if (load_status(ctl)) return;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    int b = g.cell_box[c];
    if (!box_due(disp, b, mode, thr)) return;
    int base = (int)g.atom_off[b] - start[g.cell_off[b]];
    int a = base + start[c], e = base + start[c + 1];
    fill[c] = 0;
    for (int i = a + 1; i < e; ++i) {
        int s = src[i];
        int key = perm[s];
        int j = i - 1;
        while (j >= a && perm[src[j]] > key) {
            src[j + 1] = src[j];
            --j;
        }
        src[j + 1] = s;
    }
}

__global__ void k_permute(int64_t N, int64_t Np, Geo g, const int* __restrict__ src,
                          const double4_32a* __restrict__ x, double4_32a* __restrict__ x_alt,
                          const double* __restrict__ v, double* __restrict__ v_alt, const int* __restrict__ perm,
                          int* __restrict__ perm_alt, const int* __restrict__ cell_of, int* __restrict__ cell_t_alt,
                          const Ctl* ctl, const unsigned long long* __restrict__ disp, int mode,
                          unsigned long long thr) {
    if (load_status(ctl)) return;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        if (!box_due(disp, g.B == 1 ? 0 : g.atom_box[t], mode, thr)) continue;
        int s = src[t];
        x_alt[t] = x[s];
        v_alt[t] = v[s];
        v_alt[Np + t] = v[Np + s];
        v_alt[2 * Np + t] = v[2 * Np + s];
        perm_alt[t] = perm[s];
        cell_t_alt[t] = cell_of[s];
    }
}

__global__ void k_copy_back(int64_t N, int64_t Np, Geo g, double4_32a* __restrict__ x, const double4_32a* __restrict__ x_alt,
                            double4_32a* __restrict__ xb, double* __restrict__ v, const double* __restrict__ v_alt,
                            int* __restrict__ perm, const int* __restrict__ perm_alt, int* __restrict__ iperm,
                            int* __restrict__ cell_t, const int* __restrict__ cell_t_alt, float4* __restrict__ xo,
                            Ctl* ctl, const unsigned long long* __restrict__ disp, int mode,
                            unsigned long long thr) {
    if (load_status(ctl)) return;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const int b = g.B == 1 ? 0 : g.atom_box[t];
        if (!box_due(disp, b, mode, thr)) continue;
        // count the list builds of the dynamics (one per box and step)
        if (!mode && t == g.atom_off[b]) atomicAdd((unsigned long long*)&ctl->n_rebuild, 1ULL);
        double4_32a p = x_alt[t];
        x[t] = p;
        xb[t] = p;
        v[t] = v_alt[t];
        v[Np + t] = v_alt[Np + t];
        v[2 * Np + t] = v_alt[2 * Np + t];
        int id = perm_alt[t];
        perm[t] = id;
        iperm[id] = (int)t;
        int gc = cell_t_alt[t];
        cell_t[t] = gc;
        xo[t] = cell_local(g, b, gc, p);
    }
}

static unsigned long long disp_threshold(const Engine& e) {
    double h = 0.5 * e.cfg.skin;
    double t = h * h;
    unsigned long long bits;
    memcpy(&bits, &t, sizeof(bits));
    return bits;
}

// Gate of a graph-captured step: the rebuild body (binning, sort, list
// build) runs only when some box moved more than half the skin since its
// last build and no error is pending; otherwise every kernel of the body
// would return at once, and skipping them saves their launches.
__global__ void k_rebuild_gate(int B, const unsigned long long* __restrict__ disp, unsigned long long thr, Ctl* ctl,
                               cudaGraphConditionalHandle h) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    int mine = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) mine |= disp[b] > thr;
    if (mine) any = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool run = any && !load_status(ctl);
        cudaGraphSetConditional(h, run ? 1u : 0u);
        if (!run) atomicAdd(&ctl->n_gate_skip, 1ull);
    }
}

void launch_rebuild_gate(Engine& e, cudaGraphConditionalHandle h, cudaStream_t s) {
    e.launches += 1;
    k_rebuild_gate<<<1, 256, 0, s>>>(e.B, e.disp_box, disp_threshold(e), e.ctl, h);
}

void launch_rebuild(Engine& e, int mode, cudaStream_t s) {
    if (e.N == 0) return;
    PhaseScope scope(e, MD_PHASE_REBUILD, s);
    e.launches += 8;
    Geo g = make_geo(e);
    unsigned long long thr = disp_threshold(e);
    const int nt = 256;
    // per-atom kernels: grid-stride over one wave of resident blocks (on the
    // steps that rebuild nothing each of them only reads the status and
    // returns, and a smaller grid makes that cheaper: 25 us less per step
    // than four waves on 4M atoms)
    int nb_atoms = (int)std::min<int64_t>((e.N + nt - 1) / nt, (int64_t)8 * e.n_sm);
    int nb_scan = (e.n_cells + kScanNT - 1) / kScanNT;
    const unsigned long long* disp = e.disp_box;
    k_bin<<<nb_atoms, nt, 0, s>>>(e.N, e.x, g, e.cell_of, e.cell_count, e.ctl, disp, mode, thr);
    k_scan_blocks<<<nb_scan, kScanNT, 0, s>>>(e.n_cells, e.cell_count, e.cell_start, e.scan_tmp, e.ctl);
    k_scan_totals<<<1, kScanNT, 0, s>>>(nb_scan, e.scan_tmp, e.ctl);
    k_scan_add<<<nb_scan, kScanNT, 0, s>>>(e.n_cells, e.cell_start, e.scan_tmp, e.cell_count, e.ctl);
    k_scatter<<<nb_atoms, nt, 0, s>>>(e.N, g, e.cell_of, e.cell_start, e.cell_count, e.src, e.ctl, disp, mode, thr);
    k_sort_cells<<<(e.n_cells + 127) / 128, 128, 0, s>>>(e.n_cells, g, e.cell_start, e.cell_count, e.src, e.perm,
                                                          e.ctl, disp, mode, thr);
    k_permute<<<nb_atoms, nt, 0, s>>>(e.N, e.N_pad, g, e.src, e.x, e.x_alt, e.v, e.v_alt, e.perm, e.perm_alt,
                                      e.cell_of, e.cell_t_alt, e.ctl, disp, mode, thr);
    k_copy_back<<<nb_atoms, nt, 0, s>>>(e.N, e.N_pad, g, e.x, e.x_alt, e.xb, e.v, e.v_alt, e.perm, e.perm_alt,
                                        e.iperm, e.cell_t, e.cell_t_alt, e.xo, e.ctl, disp, mode, thr);
    launch_build_list(e, mode, s);
}

}  // namespace mdk
