// Verlet neighbour-list build (Sec. 3.2, Fig. 3).
//
// The paper gives one thread block to a group of BLOCKSIZE atoms of a cell,
// one thread per atom, and walks the 27 surrounding cells in BLOCKSIZE-wide
// tiles of positions staged in shared memory. Cells of a GB300 workload hold
// ~13 atoms, so a thread per atom would leave most lanes idle on the float64
// distance test. Here one block owns one cell:
//   - the atoms of the (de-duplicated) 27-cell stencil are staged in shared
//     memory once, in stencil order;
//   - each warp takes one atom i of the cell at a time and sweeps the staged
//     candidates 32 at a time, one candidate per lane;
//   - accepted candidates are compacted with a warp ballot and a prefix
//     popcount, so the list keeps the staged order (deterministic);
//   - the list is stored column-major, nl[k * N_pad + i], so that the
//     density and force passes read it with coalesced loads.
// The test is bit-exact with the CPU oracle: d = x_j - x_i with one minimum-
// image shift, r^2 = dx*dx + dy*dy + dz*dz rounded after every operation
// (no fused multiply-add), accepted when r^2 < rl^2. A float32 prefilter
// (below) settles all candidates that are not within a proven error band of
// the list radius, so the float64 pipe is used for ~0.01 candidates per atom
// instead of ~343.
#include <algorithm>
#include <cstring>

#include "md_device.cuh"

namespace mdk {

constexpr int kNlThreads = 128;
constexpr int kNlCap = 1024;  // staged candidates per pass
constexpr int kNlMaxI = 256;  // centre-cell atoms per pass


// Lists of the atoms of cell c (one block): the stencil's atoms are staged
// in shared memory in ascending cell-id order and each warp sweeps them for
// one centre atom at a time.
__device__ __forceinline__ void build_cell_lists(int c, const Geo& g, const double4_32a* __restrict__ x,
                                                 const float4* __restrict__ xo, const int* __restrict__ cell_start,
                                                 int* __restrict__ nn, int* __restrict__ nl, int max_nb,
                                                 int64_t N_pad, double rl2, float rl2f_lo, float rl2f_hi,
                                                 bool cell_code, int& my_max) {
    __shared__ float4 so[kNlCap];
    __shared__ int sj[kNlCap];
    __shared__ int cnt[kNlMaxI];
    __shared__ int st_lo[27], st_cnt[27], st_pre[28], st_code[27];
    __shared__ float st_off[27][3];
    __shared__ int n_st;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int b = g.cell_box[c];
    const int base = (int)g.atom_off[b] - cell_start[g.cell_off[b]];
    const int xyz = g.cell_xyz[c];
    const int cc[3] = {xyz & 1023, (xyz >> 10) & 1023, (xyz >> 20) & 1023};
    const int ncx = g.nc[3 * b], ncy = g.nc[3 * b + 1], ncz = g.nc[3 * b + 2];
    const double Lx = g.L[3 * b], Ly = g.L[3 * b + 1], Lz = g.L[3 * b + 2];
    const float lfx = g.cell_len_f[3 * b], lfy = g.cell_len_f[3 * b + 1], lfz = g.cell_len_f[3 * b + 2];
    const float Lfx = (float)Lx, Lfy = (float)Ly, Lfz = (float)Lz;
    const bool wide = ncx >= 3 && ncy >= 3 && ncz >= 3;

    if (threadIdx.x < 32) {
        // one lane per stencil cell (loads in parallel), then the cells in
        // ascending id order (the rank of each id among the lanes), so every
        // list comes out sorted by neighbour slot, as stencil_sorted orders
        // them for the block-per-box schedule
        const int lane = threadIdx.x;
        const int nx = ncx >= 3 ? 3 : ncx, ny = ncy >= 3 ? 3 : ncy, nz = ncz >= 3 ? 3 : ncz;
        const int total = nx * ny * nz;
        int q = 0x7fffffff, lo = 0, cnt = 0, ox = 0, oy = 0, oz = 0, code = 0;
        if (lane < total) {
            int ix = lane / (ny * nz), iy = (lane / nz) % ny, iz = lane % nz;
            ox = ncx >= 3 ? ix - 1 : ix;
            oy = ncy >= 3 ? iy - 1 : iy;
            oz = ncz >= 3 ? iz - 1 : iz;
            int qx = (cc[0] + ox + ncx) % ncx, qy = (cc[1] + oy + ncy) % ncy, qz = (cc[2] + oz + ncz) % ncz;
            q = g.cell_rank[g.cell_off[b] + (qx * ncy + qy) * ncz + qz];
            lo = base + cell_start[q];
            cnt = base + cell_start[q + 1] - lo;
            // with 3 or more cells per axis the stencil cell's offset is the
            // minimum image, and the periodic shift is that of the wrap
            const int sx = cc[0] + ox < 0 ? -1 : (cc[0] + ox >= ncx ? 1 : 0);
            const int sy = cc[1] + oy < 0 ? -1 : (cc[1] + oy >= ncy ? 1 : 0);
            const int sz = cc[2] + oz < 0 ? -1 : (cc[2] + oz >= ncz ? 1 : 0);
            // float32 pair math (cell_code): the entry carries the cell
            // offset instead, what the mixed-precision separation needs
            code = cell_code ? make_entry(0, ox, oy, oz) : make_entry(0, sx, sy, sz);
        }
        int rank = 0;
        for (int k = 0; k < total; ++k) rank += __shfl_sync(0xffffffffu, q, k) < q;
        if (lane < total) {
            st_lo[rank] = lo;
            st_cnt[rank] = cnt;
            st_code[rank] = code;
            st_off[rank][0] = (float)ox * lfx;
            st_off[rank][1] = (float)oy * lfy;
            st_off[rank][2] = (float)oz * lfz;
        }
        __syncwarp();
        int c = lane < total ? st_cnt[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, c, o);
            if (lane >= o) c += t;
        }
        if (lane < total) st_pre[lane + 1] = c;
        if (lane == 0) {
            st_pre[0] = 0;
            n_st = total;
        }
    }
    __syncthreads();
    const int n_cand = st_pre[n_st];
    const int i_lo = base + cell_start[c], i_hi = base + cell_start[c + 1];

    for (int ib = i_lo; ib < i_hi; ib += kNlMaxI) {
        const int ni = min(kNlMaxI, i_hi - ib);
        for (int t = threadIdx.x; t < ni; t += kNlThreads) cnt[t] = 0;
        for (int cb = 0; cb < n_cand; cb += kNlCap) {
            const int nc_ = min(kNlCap, n_cand - cb);
            __syncthreads();
            for (int t = threadIdx.x; t < nc_; t += kNlThreads) {
                int q = cb + t;
                // the stencil cell holding candidate q: last k with st_pre[k] <= q
                int k = 0, hk = n_st;
                while (hk - k > 1) {
                    int mid = (k + hk) >> 1;
                    if (st_pre[mid] <= q)
                        k = mid;
                    else
                        hk = mid;
                }
                int j = st_lo[k] + (q - st_pre[k]);
                float4 o = xo[j];
                if (wide) {
                    // offset from the centre cell's origin, entry with its image
                    o.x += st_off[k][0];
                    o.y += st_off[k][1];
                    o.z += st_off[k][2];
                    j |= st_code[k];
                }
                so[t] = o;
                sj[t] = j;
            }
            __syncthreads();
            for (int ii = warp; ii < ni; ii += kNlThreads / 32) {
                const int i = ib + ii;
                const float4 oi = xo[i];
                const double4_32a xi = x[i];
                const int ci = __float_as_int(oi.w);
                const int cix = ci & 1023, ciy = (ci >> 10) & 1023, ciz = (ci >> 20) & 1023;
                int n = cnt[ii];
                for (int jb = 0; jb < nc_; jb += 32) {
                    int jj = jb + lane;
                    bool ok = false;
                    int entry = 0;
                    if (jj < nc_) {
                        if (wide) {
                            entry = sj[jj];
                            const int j = entry_slot(entry);
                            const float4 oj = so[jj];
                            const float dx = oj.x - oi.x, dy = oj.y - oi.y, dz = oj.z - oi.z;
                            const float r2f = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                            if (r2f < rl2f_lo) {
                                ok = j != i;
                            } else if (!(r2f > rl2f_hi)) {
                                int sx, sy, sz;
                                ok = exact_candidate(xi, x[j], Lx, Ly, Lz, rl2, sx, sy, sz) && j != i;
                                if (!cell_code) entry = make_entry(j, sx, sy, sz);
                            }
                        } else {
                            const int j = sj[jj];
                            int sx = 0, sy = 0, sz = 0;
                            ok = list_candidate(oi, so[jj], xi, x, j, cix, ciy, ciz, ncx, ncy, ncz, lfx, lfy, lfz,
                                                Lfx, Lfy, Lfz, Lx, Ly, Lz, rl2, rl2f_lo, rl2f_hi, sx, sy, sz) &&
                                 (j != i);
                            entry = make_entry(j, sx, sy, sz);
                        }
                    }
                    unsigned m = __ballot_sync(0xffffffffu, ok);
                    if (ok) {
                        int pos = n + __popc(m & lt_mask);
                        if (pos < max_nb) nl[(int64_t)pos * N_pad + i] = entry;
                    }
                    n += __popc(m);
                }
                if (lane == 0) cnt[ii] = n;
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ni; t += kNlThreads) {
            int n = cnt[t];
            nn[ib + t] = n;
            my_max = max(my_max, n);
        }
        __syncthreads();
    }
    __syncthreads();  // the next cell's stencil set-up overwrites st_*
}

__global__ void __launch_bounds__(kNlThreads) k_build_list(int n_cells, Geo g, const double4_32a* __restrict__ x,
                                                           const float4* __restrict__ xo,
                                                           const int* __restrict__ cell_start,
                                                           int* __restrict__ nn, int* __restrict__ nl, int max_nb,
                                                           int64_t N_pad, double rl2, float rl2f_lo, float rl2f_hi,
                                                           Ctl* ctl, const int* __restrict__ due, int mode,
                                                           bool cell_code) {
    // persistent blocks: a full build walks every cell, a partial build the
    // cells queued by k_due_cells (one block per cell at a time either way,
    // so a few boxes that rebuild still spread over the whole GPU)
    if (load_status(ctl)) return;
    int my_max = 0;
    if (mode) {
        for (int c = blockIdx.x; c < n_cells; c += gridDim.x)
            build_cell_lists(c, g, x, xo, cell_start, nn, nl, max_nb, N_pad, rl2, rl2f_lo, rl2f_hi, cell_code,
                             my_max);
    } else {
        const int n_due = ctl->n_due;
        for (int t = blockIdx.x; t < n_due; t += gridDim.x)
            build_cell_lists(due[t], g, x, xo, cell_start, nn, nl, max_nb, N_pad, rl2, rl2f_lo, rl2f_hi, cell_code,
                             my_max);
    }
    const int lane = threadIdx.x & 31;
    my_max = warp_max(my_max);
    if (lane == 0 && my_max > 0) {
        atomicMax(&ctl->max_count, my_max);
        if (my_max > max_nb) {
            atomicOr(&ctl->status, kStOverflow);
            atomicMax(&ctl->overflow_count, my_max);
        }
    }
}

// raw: the lists as built (ascending), in the reverse-index array, which
// k_build_rev overwrites next. Tiles of 32 consecutive atoms: the block
// loads the tile's rows of raw into shared memory (row k of 32 atoms is one
// 128-byte line), finds each list's split, and writes the rotated rows back
// as whole lines and each lower part as one contiguous run of nl_lo: the
// arrays of rotate_list_from, with every global access coalesced (the
// thread-per-atom form gathers one 4-byte word per lane from 32 rows).
constexpr int kRotNT = 128;
constexpr size_t kRotSmemMax = 200 * 1024;  // lists up to 1600 entries per atom

__global__ void __launch_bounds__(kRotNT) k_rotate_tiles(int64_t N, int64_t Np, Geo g, const int* __restrict__ nn,
                                                         const int* __restrict__ raw, int* __restrict__ nl,
                                                         int* __restrict__ nl_lo, int max_nb, int* __restrict__ n_up,
                                                         const Ctl* ctl, const unsigned long long* __restrict__ disp,
                                                         int mode, unsigned long long thr) {
    if (load_status(ctl)) return;
    extern __shared__ int s_tile[];  // [max_nb][32]
    __shared__ int s_lo[32];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int64_t n_tiles = (N + 31) / 32;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t i = tile * 32 + lane;
        const bool due = i < N && box_due(disp, g.B == 1 ? 0 : g.atom_box[i], mode, thr);
        // a tile none of whose atoms rebuilds is skipped by the whole block
        // (every warp holds the same 32 atoms, so the vote agrees): between
        // list builds of a batch most tiles are such tiles
        if (!__any_sync(0xffffffffu, due)) continue;
        const int n = due ? min(nn[i], max_nb) : 0;
        const int kmax = warp_max(n);
        for (int k = wq; k < kmax; k += kRotNT / 32) s_tile[k * 32 + lane] = k < n ? raw[(int64_t)k * Np + i] : 0;
        __syncthreads();
        if (wq == 0) {
            int lo = 0;
            if (n > kRotMax) {
                lo = n;  // kept ascending: the whole list is its searchable part
            } else {
                while (lo < n && entry_slot(s_tile[lo * 32 + lane]) < i) ++lo;
            }
            if (due) n_up[i] = n > kRotMax ? -1 : n - lo;
            s_lo[lane] = lo;
        }
        __syncthreads();
        // lower parts, row-major: a warp per atom, lanes along the run
        for (int a = wq; a < 32; a += kRotNT / 32) {
            const int lo = s_lo[a];
            int* out = nl_lo + (tile * 32 + a) * (int64_t)max_nb;
            for (int m = lane; m < lo; m += 32) out[m] = s_tile[m * 32 + a];
        }
        // rotated rows [upper | lower], whole lines
        const int lo = s_lo[lane];
        const bool rot = n <= kRotMax;
        for (int k = wq; k < kmax; k += kRotNT / 32) {
            if (k < n) {
                int src = k;
                if (rot) src = k + lo < n ? k + lo : k + lo - n;
                nl[(int64_t)k * Np + i] = s_tile[src * 32 + lane];
            }
        }
        __syncthreads();
    }
}

__global__ void k_rotate_lists(int64_t N, int64_t Np, Geo g, const int* __restrict__ nn,
                               const int* __restrict__ raw, int* __restrict__ nl, int* __restrict__ nl_lo,
                               int max_nb, int* __restrict__ n_up, const Ctl* ctl,
                               const unsigned long long* __restrict__ disp, int mode, unsigned long long thr) {
    if (load_status(ctl)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        if (box_due(disp, g.B == 1 ? 0 : g.atom_box[i], mode, thr))
            n_up[i] = rotate_list_from(Np, i, min(nn[i], max_nb), raw, nl, nl_lo, max_nb);
}

__global__ void k_build_rev(int64_t N, int64_t Np, Geo g, const int* __restrict__ nn, const int* __restrict__ nl,
                            const int* __restrict__ nl_lo, int max_nb, const int* __restrict__ n_up,
                            int* __restrict__ rev, const Ctl* ctl, const unsigned long long* __restrict__ disp,
                            int mode, unsigned long long thr) {
    if (load_status(ctl)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        if (box_due(disp, g.B == 1 ? 0 : g.atom_box[i], mode, thr))
            reverse_index(Np, i, min(nn[i], max_nb), n_up[i], nn, nl, nl_lo, n_up, max_nb, rev);
}

// A full rebuild restarts the largest-count record; partial rebuilds only
// raise it, so it stays an upper bound of every current list.
__global__ void k_reset_max_count(Ctl* ctl, int mode) {
    if (load_status(ctl)) return;
    ctl->n_due = 0;
    if (mode) ctl->max_count = 0;
}

// Queues the cells of the boxes whose atoms moved more than half the skin
// since their last build (one append per warp; the order of the queue does
// not matter, every cell writes its own lists).
__global__ void k_due_cells(int n_cells, Geo g, Ctl* ctl, const unsigned long long* __restrict__ disp,
                            unsigned long long thr, int* __restrict__ due) {
    if (load_status(ctl)) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const bool d = c < n_cells && disp[g.cell_box[c]] > thr;
    const unsigned m = __ballot_sync(0xffffffffu, d);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0) base = atomicAdd(&ctl->n_due, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (d) due[base + __popc(m & ((1u << lane) - 1u))] = c;
}

void launch_build_list(Engine& e, int mode, cudaStream_t s) {
    if (e.N == 0) return;
    e.launches += 2;
    Geo g = make_geo(e);
    double h = 0.5 * e.cfg.skin, t = h * h;
    unsigned long long thr;
    memcpy(&thr, &t, sizeof(thr));
    double rl2 = e.rl * e.rl;
    double margin = 4e-4 * e.rl;
    float lo = (float)(rl2 - margin), hi = (float)(rl2 + margin);
    k_reset_max_count<<<1, 1, 0, s>>>(e.ctl, mode);
    static int nl_per_sm = 0;
    if (!nl_per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nl_per_sm, k_build_list, kNlThreads, 0);
        nl_per_sm = std::max(nl_per_sm, 1);
    }
    if (!mode) {
        k_due_cells<<<(e.n_cells + 255) / 256, 256, 0, s>>>(e.n_cells, g, e.ctl, e.disp_box, thr, e.due_cells);
        e.launches += 1;
    }
    const int nl_blocks = std::max(1, std::min(e.n_cells, nl_per_sm * e.n_sm));
    // float64 lists are built into the reverse-index array and rotated from
    // there into nl (the reverse index is rebuilt right after)
    int* built = e.rev ? e.rev : e.nl;
    k_build_list<<<nl_blocks, kNlThreads, 0, s>>>(e.n_cells, g, e.x, e.xo, e.cell_start, e.nn, built, e.max_nb,
                                                  e.N_pad, rl2, lo, hi, e.ctl, e.due_cells, mode,
                                                  e.cfg.precision == MD_MIXED);
    if (e.rev) {
        // grid-stride over the atoms with four waves of resident blocks
        int nb = (int)std::min<int64_t>((e.N + 255) / 256, (int64_t)32 * e.n_sm);
        const size_t rot_smem = (size_t)e.max_nb * 32 * sizeof(int);
        if (rot_smem <= kRotSmemMax) {
            if (rot_smem > 48 * 1024)
                cudaFuncSetAttribute(k_rotate_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rot_smem);
            const int nt = (int)std::min<int64_t>((e.N + 31) / 32, (int64_t)16 * e.n_sm);
            k_rotate_tiles<<<nt, kRotNT, rot_smem, s>>>(e.N, e.N_pad, g, e.nn, e.rev, e.nl, e.nl_lo, e.max_nb,
                                                       e.n_up, e.ctl, e.disp_box, mode, thr);
        } else {
            k_rotate_lists<<<nb, 256, 0, s>>>(e.N, e.N_pad, g, e.nn, e.rev, e.nl, e.nl_lo, e.max_nb, e.n_up, e.ctl,
                                              e.disp_box, mode, thr);
        }
        k_build_rev<<<nb, 256, 0, s>>>(e.N, e.N_pad, g, e.nn, e.nl, e.nl_lo, e.max_nb, e.n_up, e.rev, e.ctl,
                                       e.disp_box, mode, thr);
        e.launches += 2;
    }
}

}  // namespace mdk
