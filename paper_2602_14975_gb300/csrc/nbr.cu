// Cell-list neighbour build (minimum image, open or periodic, batched over
// replicas). Cell grids have edge >= r_list, so all pairs lie in the 27 (or
// fewer, de-duplicated) neighbouring cells. Rows are sorted by neighbour
// index, so their order is canonical and independent of scheduling.
#include "nbr.cuh"
#include "ptx.cuh"

namespace dmts {

__device__ __forceinline__ bool gated_off(const int *gate, const int *err) {
    return (gate && *gate == 0) || *err;
}

__global__ void k_atom_rep(const int *rep_off, int n_rep, int n, int *atom_rep) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atom_rep[i] = replica_of(rep_off, n_rep, i);
}

void atom_rep_map(const int *rep_off, int n_rep, int n_atoms, int *atom_rep, cudaStream_t st) {
    if (n_atoms == 0) return;
    k_atom_rep<<<(n_atoms + 255) / 256, 256, 0, st>>>(rep_off, n_rep, n_atoms, atom_rep);
    count_launch();
}

// One block per replica: zeroes the replica's cell counts; open replicas:
// bounding box -> origin and cell edge max(r_list, extent/dim).
__global__ void k_grid_open(NbrWork w, float r_list) {
    if (gated_off(w.gate, w.err)) return;
    const int r = blockIdx.x;
    CellGrid &g = w.grid[r];
    const int nc = g.dim[0] * g.dim[1] * g.dim[2];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) w.cell_cnt[g.cell_off + c] = 0;
    if (g.box[0] > 0.f) {
        // periodic: cell counts fixed on the host; the edges follow the current box
        if (w.box && threadIdx.x == 0)
            for (int a = 0; a < 3; ++a) {
                const float L = w.box[3 * r + a];
                g.box[a] = L;
                g.inv_h[a] = (float)g.dim[a] / L;
                if (!(L * 1.000001f >= r_list * (float)g.dim[a]) || !(r_list < 0.5f * L))
                    set_error(w.err, DMTS_E_INVALID);   // the box shrank below the cell grid
            }
        return;
    }
    __shared__ float red[6][32];
    float mn[3] = {3.4e38f, 3.4e38f, 3.4e38f}, mx[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    const int beg = w.rep_off[r], end = w.rep_off[r + 1];
    for (int i = beg + threadIdx.x; i < end; i += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const float v = w.x[3 * i + a];
            mn[a] = fminf(mn[a], v);
            mx[a] = fmaxf(mx[a], v);
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(DMTS_FULL, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(DMTS_FULL, mx[a], o));
        }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) { red[a][wid] = mn[a]; red[3 + a][wid] = mx[a]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) {
            float lo = 3.4e38f, hi = -3.4e38f;
            for (int k = 0; k < nw; ++k) { lo = fminf(lo, red[a][k]); hi = fmaxf(hi, red[3 + a][k]); }
            if (end == beg) { lo = 0.f; hi = 0.f; }
            const float h = fmaxf(r_list, (hi - lo) / (float)g.dim[a]);
            g.org[a] = lo;
            g.inv_h[a] = 1.f / h;
        }
    }
}

__device__ __forceinline__ int cell_coord(float v, const CellGrid &g, int a) {
    int c;
    if (g.box[a] > 0.f) {
        const float w = v - g.box[a] * floorf(v / g.box[a]);
        c = (int)(w * g.inv_h[a]);
    } else {
        c = (int)floorf((v - g.org[a]) * g.inv_h[a]);
    }
    return min(max(c, 0), g.dim[a] - 1);
}

__global__ void k_cell_assign(NbrWork w) {
    if (gated_off(w.gate, w.err)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.n_atoms) return;
    const CellGrid g = w.grid[w.atom_rep[i]];
    const int cx = cell_coord(w.x[3 * i], g, 0), cy = cell_coord(w.x[3 * i + 1], g, 1),
              cz = cell_coord(w.x[3 * i + 2], g, 2);
    const int cell = g.cell_off + (cz * g.dim[1] + cy) * g.dim[0] + cx;
    w.atom_cell[i] = cell;
    w.atom_slot[i] = atomicAdd(&w.cell_cnt[cell], 1);
}

__global__ void k_cell_scatter(NbrWork w) {
    if (gated_off(w.gate, w.err)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.n_atoms) return;
    w.cell_atoms[w.cell_start[w.atom_cell[i]] + w.atom_slot[i]] = i;
}

// Visits every candidate j of atom i (fixed cell order, ascending j inside a
// cell); calls f(j, r2) for j != i with r2 < rc2.
template <typename Fn>
__device__ __forceinline__ void for_candidates(const NbrWork &w, int i, float rc2, Fn f) {
    const CellGrid g = w.grid[w.atom_rep[i]];
    const float xi = w.x[3 * i], yi = w.x[3 * i + 1], zi = w.x[3 * i + 2];
    const int own = w.atom_cell[i] - g.cell_off;
    const int cx = own % g.dim[0], cy = (own / g.dim[0]) % g.dim[1], cz = own / (g.dim[0] * g.dim[1]);
    int lo[3], hi[3];
    const int c3[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a) {
        if (g.box[a] > 0.f) {
            if (g.dim[a] >= 3) { lo[a] = -1; hi[a] = 1; }
            else if (g.dim[a] == 2) { lo[a] = 0; hi[a] = 1; }
            else { lo[a] = 0; hi[a] = 0; }
        } else {
            lo[a] = c3[a] > 0 ? -1 : 0;
            hi[a] = c3[a] < g.dim[a] - 1 ? 1 : 0;
        }
    }
    const float ibx = g.box[0] > 0.f ? 1.f / g.box[0] : 0.f;
    const float iby = g.box[1] > 0.f ? 1.f / g.box[1] : 0.f;
    const float ibz = g.box[2] > 0.f ? 1.f / g.box[2] : 0.f;
    for (int oz = lo[2]; oz <= hi[2]; ++oz) {
        int z = cz + oz;
        if (g.box[2] > 0.f) z = (z + g.dim[2]) % g.dim[2];
        for (int oy = lo[1]; oy <= hi[1]; ++oy) {
            int y = cy + oy;
            if (g.box[1] > 0.f) y = (y + g.dim[1]) % g.dim[1];
            for (int ox = lo[0]; ox <= hi[0]; ++ox) {
                int xx = cx + ox;
                if (g.box[0] > 0.f) xx = (xx + g.dim[0]) % g.dim[0];
                const int cell = g.cell_off + (z * g.dim[1] + y) * g.dim[0] + xx;
                const int beg = w.cell_start[cell], end = w.cell_start[cell + 1];
                for (int p = beg; p < end; ++p) {
                    const int j = w.cell_atoms[p];
                    if (j == i) continue;
                    const float dx = min_img(w.x[3 * j] - xi, g.box[0], ibx);
                    const float dy = min_img(w.x[3 * j + 1] - yi, g.box[1], iby);
                    const float dz = min_img(w.x[3 * j + 2] - zi, g.box[2], ibz);
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < rc2) f(j);
                }
            }
        }
    }
}

// Warp per atom: lanes sweep the candidates of the neighbouring cells, hits
// are collected by ballot into shared memory and written out in ascending j
// (placed by rank; a bitonic network for rows longer than 128 and in the
// fill pass without kept rows). Rows are in canonical order, so they do not
// depend on the cell layout at build time and results do not depend on when
// lists were rebuilt.
constexpr int NB_WARPS = 4;
constexpr int NB_MAXROW = 256;

// Warp sweep over the candidates of atom i. Cells are numbered x-fastest, so
// for each (z, y) row of neighbouring cells the x-run of cells is one
// contiguous range of cell_atoms (two where it wraps a periodic x boundary).
// Lane s holds range s (at most 18 for the 3 x 3 rows); the ranges are
// concatenated by a warp scan and the lanes walk the concatenation 32
// candidates at a time, so no lane idles at the end of a short cell.
template <typename Fn>
__device__ __forceinline__ void for_candidates_warp(const NbrWork &w, int i, float rc2, int lane, Fn f) {
    const CellGrid g = w.grid[w.atom_rep[i]];
    const float xi = w.x[3 * i], yi = w.x[3 * i + 1], zi = w.x[3 * i + 2];
    const int own = w.atom_cell[i] - g.cell_off;
    const int cx = own % g.dim[0], cy = (own / g.dim[0]) % g.dim[1], cz = own / (g.dim[0] * g.dim[1]);
    int lo[3], hi[3];
    const int c3[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a) {
        if (g.box[a] > 0.f) {
            if (g.dim[a] >= 3) { lo[a] = -1; hi[a] = 1; }
            else if (g.dim[a] == 2) { lo[a] = 0; hi[a] = 1; }
            else { lo[a] = 0; hi[a] = 0; }
        } else {
            lo[a] = c3[a] > 0 ? -1 : 0;
            hi[a] = c3[a] < g.dim[a] - 1 ? 1 : 0;
        }
    }
    const float ibx = g.box[0] > 0.f ? 1.f / g.box[0] : 0.f;
    const float iby = g.box[1] > 0.f ? 1.f / g.box[1] : 0.f;
    const float ibz = g.box[2] > 0.f ? 1.f / g.box[2] : 0.f;
    // x-run [x0, x1] of cells, split at a periodic wrap into [a0, b0] and [a1, b1]
    int a0 = cx + lo[0], b0 = cx + hi[0], a1 = 0, b1 = -1;
    if (a0 < 0) { a1 = a0 + g.dim[0]; b1 = g.dim[0] - 1; a0 = 0; }
    else if (b0 >= g.dim[0]) { a1 = 0; b1 = b0 - g.dim[0]; b0 = g.dim[0] - 1; }
    int seg_beg = 0, seg_len = 0, sidx = 0;
    for (int oz = lo[2]; oz <= hi[2]; ++oz) {
        int z = cz + oz;
        if (g.box[2] > 0.f) z = (z + g.dim[2]) % g.dim[2];
        for (int oy = lo[1]; oy <= hi[1]; ++oy) {
            int y = cy + oy;
            if (g.box[1] > 0.f) y = (y + g.dim[1]) % g.dim[1];
            const int row = g.cell_off + (z * g.dim[1] + y) * g.dim[0];
            if (lane == sidx) {
                seg_beg = w.cell_start[row + a0];
                seg_len = w.cell_start[row + b0 + 1] - seg_beg;
            }
            ++sidx;
            if (b1 >= a1) {
                if (lane == sidx) {
                    seg_beg = w.cell_start[row + a1];
                    seg_len = w.cell_start[row + b1 + 1] - seg_beg;
                }
                ++sidx;
            }
        }
    }
    int incl = seg_len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(DMTS_FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(DMTS_FULL, incl, 31);
    const int excl = incl - seg_len;
    for (int q0 = 0; q0 < total; q0 += 32) {
        const int q = q0 + lane;
        // range of q: the last lane whose start is <= q (starts never decrease)
        int sl = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int e = __shfl_sync(DMTS_FULL, excl, sl + st);
            if (e <= q) sl += st;
        }
        const int pb = __shfl_sync(DMTS_FULL, seg_beg, sl), pe = __shfl_sync(DMTS_FULL, excl, sl);
        bool hit = false;
        int j = -1;
        float r2 = 0.f;
        if (q < total) {
            j = w.cell_atoms[pb + (q - pe)];
            if (j != i) {
                const float dx = min_img(w.x[3 * j] - xi, g.box[0], ibx);
                const float dy = min_img(w.x[3 * j + 1] - yi, g.box[1], iby);
                const float dz = min_img(w.x[3 * j + 2] - zi, g.box[2], ibz);
                r2 = dx * dx + dy * dy + dz * dz;
                hit = r2 < rc2;
            }
        }
        f(hit, j, r2);
    }
}

constexpr unsigned SUB_FLAG = 0x80000000u;   // slot entry within the sub-list cutoff

// Ascending bitonic sort of sb[0..cnt) (values compared without SUB_FLAG).
__device__ __forceinline__ void sort_row(int *sb, int cnt, int lane) {
    int len = 32;
    while (len < cnt) len <<= 1;
    for (int t = cnt + lane; t < len; t += 32) sb[t] = 0x7fffffff;
    __syncwarp();
    for (int k = 2; k <= len; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t = lane; t < len; t += 32) {
                const int u = t ^ jj;
                if (u > t) {
                    const int a = sb[t], b = sb[u];
                    const bool up = (t & k) == 0;
                    if (((a & 0x7fffffff) > (b & 0x7fffffff)) == up) {
                        sb[t] = b;
                        sb[u] = a;
                    }
                }
            }
            __syncwarp();
        }
}

// Writes the entries of sb[0..cnt) (distinct keys, compared without
// SUB_FLAG) to dst in ascending order: each entry goes to the position given
// by the number of smaller keys. A lane ranks entries lane, lane + 32, ...;
// every key is read once per lane. cnt <= 128.
__device__ __forceinline__ void rank_scatter(const int *sb, int cnt, int *dst, int lane) {
    int v[4], k[4], r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int t = lane + 32 * q;
        v[q] = t < cnt ? sb[t] : 0;
        k[q] = t < cnt ? (v[q] & 0x7fffffff) : -1;
        r[q] = 0;
    }
#pragma unroll 4
    for (int u = 0; u < cnt; ++u) {
        const int ku = sb[u] & 0x7fffffff;
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] += ku < k[q] ? 1 : 0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (lane + 32 * q < cnt) dst[r[q]] = v[q];
}

// Row lengths (and sub-list row lengths). With w.slots the sorted row, sub
// entries flagged, is also kept for the fill, which then only copies it.
// RowAcc collects one atom's hits (warp-cooperative) and writes its counts
// and kept row.
struct RowAcc {
    int *sb;
    int cnt = 0, cnt_sub = 0;
    __device__ __forceinline__ void add(const NbrWork &w, bool keep, bool hit, int j, float r2, float rc2_sub,
                                        int lane) {
        const bool sub = hit && r2 < rc2_sub;
        const unsigned m = __ballot_sync(DMTS_FULL, hit);
        if (keep && hit) {
            const int pos = cnt + __popc(m & ((1u << lane) - 1u));
            if (pos < NB_MAXROW) sb[pos] = (int)((unsigned)j | (sub && w.counts_sub ? SUB_FLAG : 0u));
        }
        cnt += __popc(m);
        if (w.counts_sub) cnt_sub += __popc(__ballot_sync(DMTS_FULL, sub));
    }
    __device__ __forceinline__ void finish(const NbrWork &w, bool keep, int i, int lane) {
        if (lane == 0) {
            w.counts[i] = cnt;
            if (w.counts_sub) w.counts_sub[i] = cnt_sub;
        }
        if (keep && cnt <= w.slot_cap && cnt <= NB_MAXROW) {
            __syncwarp();
            int *dst = w.slots + (size_t)i * w.slot_cap;
            if (cnt <= 128) {
                rank_scatter(sb, cnt, dst, lane);
            } else {
                sort_row(sb, cnt, lane);
                for (int t = lane; t < cnt; t += 32) dst[t] = sb[t];
            }
        }
        __syncwarp();
    }
};

__global__ void __launch_bounds__(NB_WARPS * 32) k_nbr_count_warp(NbrWork w, float rc2, float rc2_sub) {
    if (gated_off(w.gate, w.err)) return;
    __shared__ int buf[NB_WARPS][NB_MAXROW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * NB_WARPS + warp;
    if (i >= w.n_atoms) return;
    const bool keep = w.slots != nullptr;
    RowAcc acc{buf[warp]};
    for_candidates_warp(w, i, rc2, lane, [&](bool hit, int j, float r2) { acc.add(w, keep, hit, j, r2, rc2_sub, lane); });
    acc.finish(w, keep, i, lane);
}

// The same count by cells: one block per cell stages the indices and
// positions of every candidate of its neighbouring cells in shared memory
// once (in the order for_candidates_warp visits them), then each warp
// sweeps them for one atom of the cell at a time. The candidates' positions
// are exact copies, so every distance and decision is the same as in the
// per-atom sweep; a cell with more candidates than fit falls back to it.
constexpr int NBC_WARPS = 8, NBC_CAP = 2048;

__global__ void __launch_bounds__(NBC_WARPS * 32) k_nbr_count_cell(NbrWork w, float rc2, float rc2_sub) {
    if (gated_off(w.gate, w.err)) return;
    __shared__ int cj[NBC_CAP];
    __shared__ float cx[NBC_CAP], cy[NBC_CAP], cz[NBC_CAP];
    __shared__ int buf[NBC_WARPS][NB_MAXROW];
    __shared__ int seg_beg[18], seg_excl[19];
    const int c = blockIdx.x;
    const int a_beg = w.cell_start[c], a_end = w.cell_start[c + 1];
    if (a_beg == a_end) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const CellGrid g = w.grid[w.atom_rep[w.cell_atoms[a_beg]]];
    if (threadIdx.x == 0) {
        // the neighbouring cells' x-runs, as for_candidates_warp forms them
        const int own = c - g.cell_off;
        const int ccx = own % g.dim[0], ccy = (own / g.dim[0]) % g.dim[1], ccz = own / (g.dim[0] * g.dim[1]);
        int lo[3], hi[3];
        const int c3[3] = {ccx, ccy, ccz};
        for (int a = 0; a < 3; ++a) {
            if (g.box[a] > 0.f) {
                if (g.dim[a] >= 3) { lo[a] = -1; hi[a] = 1; }
                else if (g.dim[a] == 2) { lo[a] = 0; hi[a] = 1; }
                else { lo[a] = 0; hi[a] = 0; }
            } else {
                lo[a] = c3[a] > 0 ? -1 : 0;
                hi[a] = c3[a] < g.dim[a] - 1 ? 1 : 0;
            }
        }
        int a0 = ccx + lo[0], b0 = ccx + hi[0], a1 = 0, b1 = -1;
        if (a0 < 0) { a1 = a0 + g.dim[0]; b1 = g.dim[0] - 1; a0 = 0; }
        else if (b0 >= g.dim[0]) { a1 = 0; b1 = b0 - g.dim[0]; b0 = g.dim[0] - 1; }
        int ns = 0, tot = 0;
        for (int oz = lo[2]; oz <= hi[2]; ++oz) {
            int z = ccz + oz;
            if (g.box[2] > 0.f) z = (z + g.dim[2]) % g.dim[2];
            for (int oy = lo[1]; oy <= hi[1]; ++oy) {
                int y = ccy + oy;
                if (g.box[1] > 0.f) y = (y + g.dim[1]) % g.dim[1];
                const int row = g.cell_off + (z * g.dim[1] + y) * g.dim[0];
                seg_beg[ns] = w.cell_start[row + a0];
                seg_excl[ns] = tot;
                tot += w.cell_start[row + b0 + 1] - seg_beg[ns];
                ++ns;
                if (b1 >= a1) {
                    seg_beg[ns] = w.cell_start[row + a1];
                    seg_excl[ns] = tot;
                    tot += w.cell_start[row + b1 + 1] - seg_beg[ns];
                    ++ns;
                }
            }
        }
        for (int k = ns; k < 19; ++k) seg_excl[k] = tot;
    }
    __syncthreads();
    const int total = seg_excl[18];
    const bool staged = total <= NBC_CAP;
    if (staged) {
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            int sl = 0;
            while (seg_excl[sl + 1] <= q) ++sl;
            const int j = w.cell_atoms[seg_beg[sl] + (q - seg_excl[sl])];
            cj[q] = j;
            cx[q] = w.x[3 * j];
            cy[q] = w.x[3 * j + 1];
            cz[q] = w.x[3 * j + 2];
        }
    }
    __syncthreads();
    const bool keep = w.slots != nullptr;
    const float ibx = g.box[0] > 0.f ? 1.f / g.box[0] : 0.f;
    const float iby = g.box[1] > 0.f ? 1.f / g.box[1] : 0.f;
    const float ibz = g.box[2] > 0.f ? 1.f / g.box[2] : 0.f;
    for (int k = a_beg + warp; k < a_end; k += NBC_WARPS) {
        const int i = w.cell_atoms[k];
        RowAcc acc{buf[warp]};
        if (staged) {
            const float xi = w.x[3 * i], yi = w.x[3 * i + 1], zi = w.x[3 * i + 2];
            for (int q0 = 0; q0 < total; q0 += 32) {
                const int q = q0 + lane;
                bool hit = false;
                int j = -1;
                float r2 = 0.f;
                if (q < total) {
                    j = cj[q];
                    if (j != i) {
                        const float dx = min_img(cx[q] - xi, g.box[0], ibx);
                        const float dy = min_img(cy[q] - yi, g.box[1], iby);
                        const float dz = min_img(cz[q] - zi, g.box[2], ibz);
                        r2 = dx * dx + dy * dy + dz * dz;
                        hit = r2 < rc2;
                    }
                }
                acc.add(w, keep, hit, j, r2, rc2_sub, lane);
            }
        } else {
            for_candidates_warp(w, i, rc2, lane,
                                [&](bool hit, int j, float r2) { acc.add(w, keep, hit, j, r2, rc2_sub, lane); });
        }
        acc.finish(w, keep, i, lane);
    }
}

// Appends, in order, the entries of the sorted row src[0..n) within rc2_sub
// to dst (warp-cooperative; distances recomputed exactly as in the build).
__device__ __forceinline__ void write_sub_row(const NbrWork &w, int i, const int *src, int n, float rc2_sub,
                                              int *dst, int lane) {
    const CellGrid g = w.grid[w.atom_rep[i]];
    const float ibx = g.box[0] > 0.f ? 1.f / g.box[0] : 0.f, iby = g.box[1] > 0.f ? 1.f / g.box[1] : 0.f,
                ibz = g.box[2] > 0.f ? 1.f / g.box[2] : 0.f;
    const float xi = w.x[3 * i], yi = w.x[3 * i + 1], zi = w.x[3 * i + 2];
    int done = 0;
    for (int t0 = 0; t0 < n; t0 += 32) {
        const int t = t0 + lane;
        bool keep = false;
        int j = 0;
        if (t < n) {
            j = src[t];
            const float dx = min_img(w.x[3 * j] - xi, g.box[0], ibx);
            const float dy = min_img(w.x[3 * j + 1] - yi, g.box[1], iby);
            const float dz = min_img(w.x[3 * j + 2] - zi, g.box[2], ibz);
            keep = dx * dx + dy * dy + dz * dz < rc2_sub;
        }
        const unsigned m = __ballot_sync(DMTS_FULL, keep);
        if (keep) dst[done + __popc(m & ((1u << lane) - 1u))] = j;
        done += __popc(m);
    }
}

__global__ void __launch_bounds__(NB_WARPS * 32) k_nbr_fill_warp(NbrWork w, float rc2, const int *row_ptr, int *col,
                                                                 float *x_ref, float rc2_sub, const int *sub_row,
                                                                 int *sub_col) {
    if (gated_off(w.gate, w.err)) return;
    __shared__ int buf[NB_WARPS][NB_MAXROW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * NB_WARPS + warp;
    if (i >= w.n_atoms) return;
    int *sb = buf[warp];
    const int beg = row_ptr[i], n = row_ptr[i + 1] - beg;
    if (w.slots && n <= w.slot_cap && n <= NB_MAXROW) {
        // the count pass kept the sorted row: copy it, sub entries by their flag
        const int *src = w.slots + (size_t)i * w.slot_cap;
        int done = 0;
        for (int t0 = 0; t0 < n; t0 += 32) {
            const int t = t0 + lane;
            const unsigned v = t < n ? (unsigned)src[t] : 0u;
            const int j = (int)(v & ~SUB_FLAG);
            if (t < n) col[beg + t] = j;
            if (sub_col) {
                const bool in = t < n && (v & SUB_FLAG);
                const unsigned m = __ballot_sync(DMTS_FULL, in);
                if (in) sub_col[sub_row[i] + done + __popc(m & ((1u << lane) - 1u))] = j;
                done += __popc(m);
            }
        }
    } else if (n <= NB_MAXROW) {
        int cnt = 0;
        for_candidates_warp(w, i, rc2, lane, [&](bool hit, int j, float) {
            const unsigned m = __ballot_sync(DMTS_FULL, hit);
            if (hit) sb[cnt + __popc(m & ((1u << lane) - 1u))] = j;
            cnt += __popc(m);
        });
        sort_row(sb, cnt, lane);
        for (int t = lane; t < cnt; t += 32) col[beg + t] = sb[t];
        if (sub_col) write_sub_row(w, i, sb, cnt, rc2_sub, sub_col + sub_row[i], lane);
    } else {
        // rows longer than the shared buffer: serial fill + insertion sort
        if (lane == 0) {
            int p = beg;
            for_candidates(w, i, rc2, [&](int j) { col[p++] = j; });
            for (int a = beg + 1; a < p; ++a) {
                const int v = col[a];
                int b = a - 1;
                while (b >= beg && col[b] > v) {
                    col[b + 1] = col[b];
                    --b;
                }
                col[b + 1] = v;
            }
        }
        __syncwarp();
        if (sub_col) write_sub_row(w, i, col + beg, n, rc2_sub, sub_col + sub_row[i], lane);
    }
    if (x_ref && lane == 0) {
        x_ref[3 * i] = w.x[3 * i];
        x_ref[3 * i + 1] = w.x[3 * i + 1];
        x_ref[3 * i + 2] = w.x[3 * i + 2];
    }
}

// ------------------------------------------------------------ prefix scan
// Decoupled look-back: each block takes the next tile in order (a counter,
// so that every tile's predecessors have started), sums its kScanTile
// elements, publishes that sum, and walks back over its predecessors'
// published words until one carries a full prefix; then it publishes its
// own prefix and writes its outputs. A status word packs (launch tag, flag,
// value): 28 bits of tag, 2 of flag (1 = tile sum, 2 = prefix), 34 of value,
// so words left by earlier scans never look valid.
constexpr int SCAN_THREADS = 256, SCAN_ITEMS = kScanTile / SCAN_THREADS;
constexpr int kFlagSum = 1, kFlagPrefix = 2;

__device__ __forceinline__ unsigned long long scan_word(unsigned tag, int flag, long long v) {
    return ((unsigned long long)(tag & 0x0fffffffu) << 36) | ((unsigned long long)flag << 34) |
           ((unsigned long long)v & 0x3ffffffffull);
}

struct ScanJob {
    const int *in;
    int *out;
    long long cap;
    long long *total;
};

__global__ void __launch_bounds__(SCAN_THREADS) k_scan(ScanJob j0, ScanJob j1, int n, int n_tiles,
                                                       unsigned long long *status_all, unsigned long long *counters,
                                                       int tiles_cap, int *err, const int *gate) {
    if (gated_off(gate, err)) return;
    const ScanJob J = blockIdx.y ? j1 : j0;
    unsigned long long *status = status_all + (size_t)blockIdx.y * tiles_cap;
    unsigned long long *counter = counters + blockIdx.y;
    __shared__ int tile_sh;
    __shared__ unsigned tag_sh;
    __shared__ long long warp_tot[SCAN_THREADS / 32], excl_sh;
    if (threadIdx.x == 0) {
        // every block of this launch takes one tile and reads the same epoch;
        // the block that takes the last one opens the next epoch
        const unsigned long long old = atomicAdd(counter, 1ull);
        const int t = (int)(old & 0xffffffffull);
        const unsigned epoch = (unsigned)(old >> 32);
        if (t == n_tiles - 1) atomicExch(counter, (unsigned long long)(epoch + 1u) << 32);
        tile_sh = t;
        tag_sh = epoch % 0x0ffffffeu + 1u;   // 1 .. 2^28 - 2: zeroed words carry tag 0
    }
    __syncthreads();
    const unsigned tag = tag_sh;
    const int tile = tile_sh, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int first = tile * kScanTile + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = first + k < n ? J.in[first + k] : 0;
        s += v[k];
    }
    // block-wide inclusive scan of the per-thread sums
    long long inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(DMTS_FULL, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    long long wbase = 0, agg = 0;
#pragma unroll
    for (int w = 0; w < SCAN_THREADS / 32; ++w) {
        if (w < wid) wbase += warp_tot[w];
        agg += warp_tot[w];
    }
    const long long mine = wbase + inc - s;   // exclusive prefix of this thread inside the tile
    if (threadIdx.x == 0) {
        long long excl = 0;
        volatile unsigned long long *vs = status;
        if (tile == 0) {
            vs[0] = scan_word(tag, kFlagPrefix, agg);
        } else {
            vs[tile] = scan_word(tag, kFlagSum, agg);
            const uint64_t t0 = globaltimer_ns();
            for (int p = tile - 1; p >= 0;) {
                const unsigned long long wd = vs[p];
                const int flag = (int)((wd >> 34) & 3ull);
                if ((unsigned)(wd >> 36) != (tag & 0x0fffffffu) || flag == 0) {
                    if (globaltimer_ns() - t0 > kWaitLimitNs) {   // a predecessor never published
                        set_error(err, DMTS_E_TIMEOUT);
                        excl = -1;
                        break;
                    }
                    continue;
                }
                excl += (long long)(wd & 0x3ffffffffull);
                if (flag == kFlagPrefix) break;
                --p;
            }
            if (excl >= 0) vs[tile] = scan_word(tag, kFlagPrefix, excl + agg);
        }
        excl_sh = excl;
    }
    __syncthreads();
    const long long excl = excl_sh;
    if (excl < 0) return;
    long long run = excl + mine;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (first + k < n) J.out[first + k] = (int)run;
        run += v[k];
    }
    if (tile == n_tiles - 1 && threadIdx.x == 0) {
        const long long tot = excl + agg;
        J.out[n] = (int)tot;
        if (J.total) *J.total = tot;
        if ((J.cap >= 0 && tot > J.cap) || tot > 0x7fffffffLL) set_error(err, DMTS_E_NBR_OVERFLOW);
    }
}

void scan_ints(const NbrWork &w, const int *in0, int *out0, long long cap0, long long *total0, const int *in1,
               int *out1, long long cap1, long long *total1, int n, cudaStream_t st) {
    const int tiles = (n + kScanTile - 1) / kScanTile;
    const int n_tiles = tiles > 0 ? tiles : 1;
    dim3 grid(n_tiles, in1 ? 2 : 1);
    k_scan<<<grid, SCAN_THREADS, 0, st>>>(ScanJob{in0, out0, cap0, total0}, ScanJob{in1, out1, cap1, total1}, n,
                                          n_tiles, w.scan_status, w.scan_counter, w.scan_tiles, w.err, w.gate);
    count_launch();
}

void nbr_cells(const NbrWork &w, float r_list, cudaStream_t st) {
    if (w.n_atoms == 0) return;
    k_grid_open<<<w.n_rep, 256, 0, st>>>(w, r_list);
    count_launch();
    const int nb = (w.n_atoms + 255) / 256;
    k_cell_assign<<<nb, 256, 0, st>>>(w);
    count_launch();
    scan_ints(w, w.cell_cnt, w.cell_start, -1, nullptr, nullptr, nullptr, -1, nullptr, w.n_cells, st);
    k_cell_scatter<<<nb, 256, 0, st>>>(w);
    count_launch();
}

void nbr_fill(const NbrWork &w, float r_list, int *row_ptr, int *col, long long capacity, float *x_ref,
              cudaStream_t st, float r_sub, int *sub_row, int *sub_col, long long sub_capacity) {
    if (w.n_atoms == 0) return;
    const int nb = (w.n_atoms + NB_WARPS - 1) / NB_WARPS;
    NbrWork wc = w;
    if (!sub_row) wc.counts_sub = nullptr;
    k_nbr_count_cell<<<wc.n_cells, NBC_WARPS * 32, 0, st>>>(wc, r_list * r_list, r_sub * r_sub);
    count_launch();
    // the full list's and the sub-list's row offsets in one launch
    scan_ints(wc, wc.counts, row_ptr, capacity, wc.total, wc.counts_sub, wc.counts_sub ? sub_row : nullptr,
              sub_capacity, nullptr, wc.n_atoms, st);
    if (col) {
        k_nbr_fill_warp<<<nb, NB_WARPS * 32, 0, st>>>(wc, r_list * r_list, row_ptr, col, x_ref, r_sub * r_sub,
                                                      wc.counts_sub ? sub_row : nullptr,
                                                      wc.counts_sub ? sub_col : nullptr);
        count_launch();
    }
}

}  // namespace dmts
