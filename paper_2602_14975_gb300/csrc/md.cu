// NC direct-force head (Sec. 2 "Model architecture"), the bonded + LJ prior,
// and the fused BAOAB/RESPA integrator with Philox4x32-10 noise (Algorithm 1).
#include "md.cuh"

namespace dmts {

// ---------------------------------------------------------- node helpers
__global__ void k_embed(int n, int C, const uint8_t *species, const float *emb, float *s) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C) return;
    const int i = (int)(idx / C), c = (int)(idx % C);
    s[idx] = emb[species[i] * C + c];
}

void launch_embed(int n, int C, const uint8_t *species, const float *emb, float *s, cudaStream_t st) {
    if (n == 0) return;
    const size_t tot = (size_t)n * C;
    k_embed<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, C, species, emb, s);
}

// e_atom[i] = scale * sum_c u[i][c]  (warp per atom)
__global__ void k_rowsum(int n, int C, const float *u, float scale, float *e_atom) {
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    float s = 0.f;
    for (int c = lane; c < C; c += 32) s += u[(size_t)i * C + c];
    s = warp_sum(s);
    if (lane == 0) e_atom[i] = scale * s;
}

void launch_rowsum(int n, int C, const float *u, float scale, float *e_atom, cudaStream_t st) {
    if (n == 0) return;
    k_rowsum<<<(n + 7) / 8, 256, 0, st>>>(n, C, u, scale, e_atom);
}

// V[i][h][a] = sum_c U[h][c] A[i][1+a][c]   (vector part of tensor head h)
__global__ void k_nc_vectors(int n, int C, int n_l, const float *A, const float *U, float *V, const int *err) {
    if (*err) return;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    for (int h = 0; h < n_l; ++h)
        for (int a = 0; a < 3; ++a) {
            float s = 0.f;
            for (int c = lane; c < C; c += 32) s += U[h * C + c] * A[((size_t)i * 4 + 1 + a) * C + c];
            s = warp_sum(s);
            if (lane == 0) V[((size_t)i * n_l + h) * 3 + a] = s;
        }
}

void launch_nc_vectors(int n, int C, int n_l, const float *A, const float *U, float *V, const int *err,
                       cudaStream_t st) {
    if (n == 0) return;
    k_nc_vectors<<<(n + 7) / 8, 256, 0, st>>>(n, C, n_l, A, U, V, err);
}

__device__ __forceinline__ void bond_force(const BondTable &b, const float *x, int a, float bx, float by,
                                           float bz, float ibx, float iby, float ibz, int lane, float &fx,
                                           float &fy, float &fz, float &e) {
    const float xa = x[3 * a], ya = x[3 * a + 1], za = x[3 * a + 2];
    for (int q = b.ptr[a] + lane; q < b.ptr[a + 1]; q += 32) {
        const int j = b.idx[q];
        const float dx = min_img(x[3 * j] - xa, bx, ibx);
        const float dy = min_img(x[3 * j + 1] - ya, by, iby);
        const float dz = min_img(x[3 * j + 2] - za, bz, ibz);
        const float r = sqrtf(dx * dx + dy * dy + dz * dz);
        const float dr = r - b.r0[q];
        const float g = b.k * dr / r;     // F_a = k (r - r0) d / r, d = x_j - x_a
        fx += g * dx; fy += g * dy; fz += g * dz;
        e += 0.25f * b.k * dr * dr;       // each bond is listed by both atoms
    }
}

// Visits the active entries of a neighbour row (those with pred(j) true)
// such that the g-th active entry, in row order, is handled by lane g % 32.
// Which lane sums which edge then depends only on the active edges, not on
// the extra skin entries a list happens to hold, so warp-level sums are
// reproducible whenever the list was rebuilt. fn(j) runs on the owning lane.
template <typename Pred, typename Fn>
__device__ __forceinline__ void for_active_canonical(const int *col, int beg, int end, int *queue, int lane,
                                                     Pred pred, Fn fn) {
    int queued = 0, taken = 0;
    for (int base = beg; base < end; base += 32) {
        const int e = base + lane;
        const int j = e < end ? col[e] : -1;
        const bool act = j >= 0 && pred(j);
        const unsigned m = __ballot_sync(DMTS_FULL, act);
        if (act) queue[(queued + __popc(m & ((1u << lane) - 1u))) & 63] = j;
        queued += __popc(m);
        __syncwarp();
        if (queued - taken >= 32) {
            fn(queue[(taken + lane) & 63]);
            taken += 32;
        }
        __syncwarp();
    }
    if (taken + lane < queued) fn(queue[(taken + lane) & 63]);
    __syncwarp();
}

__device__ __forceinline__ bool is_bonded(const BondTable &b, int a, int j) {
    for (int q = b.ptr[a]; q < b.ptr[a + 1]; ++q)
        if (b.idx[q] == j) return true;
    return false;
}

// Screened nuclear repulsion of one pair (ZBL universal screening, switched
// off by the envelope): returns E and writes dE/dr.
__device__ __forceinline__ float rep_pair(const RepTable &t, int si, int sj, float r, float *dEdr) {
    const float zz = t.zz[si][sj], ia = t.inv_a[si][sj];
    const float xs = r * ia;
    const float e0 = expf(-3.19980f * xs), e1 = expf(-0.94229f * xs), e2 = expf(-0.40290f * xs),
                e3 = expf(-0.20162f * xs);
    const float phi = 0.18175f * e0 + 0.50986f * e1 + 0.28022f * e2 + 0.02817f * e3;
    const float dphi = -(0.18175f * 3.19980f * e0 + 0.50986f * 0.94229f * e1 + 0.28022f * 0.40290f * e2 +
                         0.02817f * 0.20162f * e3);
    float du;
    const float fc = envelope(r * t.inv_rc, t.p, &du);
    const float ir = 1.f / r;
    const float E0 = zz * ir * phi;
    const float dE0 = -E0 * ir + zz * ir * dphi * ia;
    *dEdr = dE0 * fc + E0 * du * t.inv_rc;
    return E0 * fc;
}

// ------------------------------------------------------------- NC head
// Warp per atom a; lane per neighbour j. For each head h:
//   c_ajh = q_ah . k_jh / sqrt(n_c),  c_jah = q_jh . k_ah / sqrt(n_c)
//   F_aj = (sum_{h<K} c_ajh B_h) (n + sum_{h<n_l} c_aj(K+h) V_ah) f_c
//   F_ja = (sum_{h<K} c_jah B_h) (-n + sum_{h<n_l} c_ja(K+h) V_jh) f_c
//   F_a = scale sum_j (F_aj - F_ja) (+ bonds)
template <int K, int NC, int NL>
__global__ void __launch_bounds__(128) k_nc_head(NCHeadArgs g) {
    constexpr int H = K + NL, QKW = 2 * H * NC;
    __shared__ float sh_qk[4][QKW];
    __shared__ float sh_v[4][NL * 3];
    __shared__ int sh_queue[4][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wa = blockIdx.x * 4 + warp;
    if (wa >= g.n_atoms || *g.err) return;
    const int a = g.order ? __ldg(g.order + wa) : wa;
    for (int t = lane; t < QKW; t += 32) sh_qk[warp][t] = g.QK[(size_t)a * QKW + t];
    for (int t = lane; t < NL * 3; t += 32) sh_v[warp][t] = g.V[(size_t)a * NL * 3 + t];
    __syncwarp();
    const float *qa = sh_qk[warp], *ka = sh_qk[warp] + H * NC, *va = sh_v[warp];
    const int rep = g.atom_rep[a];
    const float bx = g.box[3 * rep], by = g.box[3 * rep + 1], bz = g.box[3 * rep + 2];
    const float ibx = bx > 0.f ? 1.f / bx : 0.f, iby = by > 0.f ? 1.f / by : 0.f, ibz = bz > 0.f ? 1.f / bz : 0.f;
    const float xa = g.x[3 * a], ya = g.x[3 * a + 1], za = g.x[3 * a + 2];
    const float rc2 = g.rc * g.rc, isnc = rsqrtf((float)NC);
    const bool with_rep = g.bonds.ptr && g.rep.on;
    const float rep2 = g.rep.rc * g.rep.rc;
    const int sa = g.species[a];
    float fx = 0.f, fy = 0.f, fz = 0.f, rx = 0.f, ry = 0.f, rz = 0.f;
    auto disp = [&](int j, float &dx, float &dy, float &dz) {
        dx = min_img(__ldg(g.x + 3 * j) - xa, bx, ibx);
        dy = min_img(__ldg(g.x + 3 * j + 1) - ya, by, iby);
        dz = min_img(__ldg(g.x + 3 * j + 2) - za, bz, ibz);
    };
    auto active = [&](int j) {
        float dx, dy, dz;
        disp(j, dx, dy, dz);
        return dx * dx + dy * dy + dz * dz < rc2;
    };
    auto edge = [&](int j) {
        float dx, dy, dz;
        disp(j, dx, dy, dz);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float r = sqrtf(r2), inv = 1.f / r;
        if (with_rep && r2 < rep2 && !is_bonded(g.bonds, a, j)) {
            float dE;
            rep_pair(g.rep, sa, g.species[j], r, &dE);
            const float c = dE * inv;              // F_a = E'(r) d / r
            rx += c * dx; ry += c * dy; rz += c * dz;
        }
        const float nx = dx * inv, ny = dy * inv, nz = dz * inv;
        float du;
        const float fc = envelope(r * g.inv_rc, g.p, &du);
        float B[K];
        bessel<K, false>(r, g.inv_rc, g.bnorm, B, nullptr);
        const float4 *qj4 = reinterpret_cast<const float4 *>(g.QK + (size_t)j * QKW);
        const float4 *kj4 = qj4 + H * NC / 4;
        float Saj = 0.f, Sja = 0.f;
        float vax = 0.f, vay = 0.f, vaz = 0.f, vjx = 0.f, vjy = 0.f, vjz = 0.f;
#pragma unroll
        for (int h = 0; h < H; ++h) {
            float caj = 0.f, cja = 0.f;
#pragma unroll
            for (int q = 0; q < NC / 4; ++q) {
                const float4 kj = __ldg(kj4 + h * NC / 4 + q);
                const float4 qj = __ldg(qj4 + h * NC / 4 + q);
                const float *qah = qa + h * NC + 4 * q, *kah = ka + h * NC + 4 * q;
                caj = fmaf(qah[0], kj.x, fmaf(qah[1], kj.y, fmaf(qah[2], kj.z, fmaf(qah[3], kj.w, caj))));
                cja = fmaf(qj.x, kah[0], fmaf(qj.y, kah[1], fmaf(qj.z, kah[2], fmaf(qj.w, kah[3], cja))));
            }
            caj *= isnc;
            cja *= isnc;
            if (h < K) {
                Saj = fmaf(caj, B[h], Saj);
                Sja = fmaf(cja, B[h], Sja);
            } else {
                const int t = h - K;
                vax = fmaf(caj, va[3 * t], vax);
                vay = fmaf(caj, va[3 * t + 1], vay);
                vaz = fmaf(caj, va[3 * t + 2], vaz);
                const float *vj = g.V + ((size_t)j * NL + t) * 3;
                vjx = fmaf(cja, __ldg(vj), vjx);
                vjy = fmaf(cja, __ldg(vj + 1), vjy);
                vjz = fmaf(cja, __ldg(vj + 2), vjz);
            }
        }
        const float pa = Saj * fc, pj = Sja * fc;
        fx += pa * (nx + vax) - pj * (-nx + vjx);
        fy += pa * (ny + vay) - pj * (-ny + vjy);
        fz += pa * (nz + vaz) - pj * (-nz + vjz);
    };
    for_active_canonical(g.col, g.row_ptr[a], g.row_ptr[a + 1], sh_queue[warp], lane, active, edge);
    fx = fmaf(g.scale, fx, rx); fy = fmaf(g.scale, fy, ry); fz = fmaf(g.scale, fz, rz);
    if (g.bonds.ptr) {
        float e = 0.f;
        bond_force(g.bonds, g.x, a, bx, by, bz, ibx, iby, ibz, lane, fx, fy, fz, e);
    }
    fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz);
    if (lane == 0) {
        g.F[3 * a] = fx; g.F[3 * a + 1] = fy; g.F[3 * a + 2] = fz;
    }
}

void launch_nc_head(int K, int n_c, int n_l, const NCHeadArgs &a, cudaStream_t st) {
    if (a.n_atoms == 0) return;
    const int blocks = (a.n_atoms + 3) / 4;
    if (K == 8 && n_c == 8 && n_l == 2) k_nc_head<8, 8, 2><<<blocks, 128, 0, st>>>(a);
    else if (K == 8 && n_c == 8 && n_l == 1) k_nc_head<8, 8, 1><<<blocks, 128, 0, st>>>(a);
    else if (K == 8 && n_c == 8 && n_l == 3) k_nc_head<8, 8, 3><<<blocks, 128, 0, st>>>(a);
    else if (K == 8 && n_c == 8 && n_l == 4) k_nc_head<8, 8, 4><<<blocks, 128, 0, st>>>(a);
}

// Block per replica: FP64 sum (of fp32 batch sums of eight atoms) of F_in
// over the replica, then subtract the mean.
__global__ void k_mean_sub(const float *__restrict__ F_in, float *__restrict__ F_out, const int *__restrict__ rep_off,
                           double *__restrict__ net, const int *__restrict__ err) {
    if (*err) return;
    __shared__ double red[3][32];
    __shared__ double mean[3];
    const int r = blockIdx.x;
    const int beg = rep_off[r], end = rep_off[r + 1];
    double s[3] = {0.0, 0.0, 0.0};
    // eight independent loads in flight per thread, then the FP64 adds in order
    const int stride = blockDim.x;
    for (int i0 = beg + threadIdx.x; i0 < end; i0 += 8 * stride) {
        float v[8][3];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * stride;
            for (int a = 0; a < 3; ++a) v[u][a] = i < end ? F_in[3 * i + a] : 0.f;
        }
        // batch of eight summed in fp32, batch sums accumulated in fp64 (the
        // fp64 units are few on this GPU: this keeps one block per replica fast)
        float b[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int u = 0; u < 8; ++u)
            for (int a = 0; a < 3; ++a) b[a] += v[u][a];
        for (int a = 0; a < 3; ++a) s[a] += (double)b[a];
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int a = 0; a < 3; ++a) {
        s[a] = warp_sum_d(s[a]);
        if (lane == 0) red[a][wid] = s[a];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int k = 0; k < nw; ++k) t += red[threadIdx.x][k];
        if (net) net[3 * r + threadIdx.x] = t;
        mean[threadIdx.x] = end > beg ? t / (double)(end - beg) : 0.0;
    }
    __syncthreads();
    const float mx = (float)mean[0], my = (float)mean[1], mz = (float)mean[2];
    for (int i0 = beg + threadIdx.x; i0 < end; i0 += 8 * stride) {
        float v[8][3];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * stride;
            for (int a = 0; a < 3; ++a) v[u][a] = i < end ? F_in[3 * i + a] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * stride;
            if (i < end) {
                F_out[3 * i] = v[u][0] - mx;
                F_out[3 * i + 1] = v[u][1] - my;
                F_out[3 * i + 2] = v[u][2] - mz;
            }
        }
    }
}

void launch_mean_sub(const float *F_in, float *F_out, const int *rep_off, int n_rep, double *net,
                     const int *err, cudaStream_t st) {
    if (n_rep == 0) return;
    k_mean_sub<<<n_rep, 1024, 0, st>>>(F_in, F_out, rep_off, net, err);
}

// ---------------------------------------------------------------- prior
// Warp per atom over its neighbour row: screened repulsion between pairs that
// are not bonded; LJ between heavy atoms of different molecules,
// 4 eps ((s/r)^12 - (s/r)^6) f(r/lj_rc; p); plus bonds.
__global__ void __launch_bounds__(128) k_prior(PriorArgs g) {
    __shared__ int sh_queue[4][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wa = blockIdx.x * 4 + warp;
    if (wa >= g.n_atoms || *g.err) return;
    const int a = g.order ? __ldg(g.order + wa) : wa;
    const int rep = g.atom_rep[a];
    const float bx = g.box[3 * rep], by = g.box[3 * rep + 1], bz = g.box[3 * rep + 2];
    const float ibx = bx > 0.f ? 1.f / bx : 0.f, iby = by > 0.f ? 1.f / by : 0.f, ibz = bz > 0.f ? 1.f / bz : 0.f;
    const float xa = g.x[3 * a], ya = g.x[3 * a + 1], za = g.x[3 * a + 2];
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    const int sa = g.species[a], ma = g.mol_id[a];
    const float rc2 = g.lj_rc * g.lj_rc, inv_rc = 1.f / g.lj_rc, s2 = g.lj_sigma * g.lj_sigma;
    const float rep2 = g.rep.on ? g.rep.rc * g.rep.rc : 0.f;
    const float cut2 = fmaxf(rc2, rep2);
    auto disp = [&](int j, float &dx, float &dy, float &dz) {
        dx = min_img(g.x[3 * j] - xa, bx, ibx);
        dy = min_img(g.x[3 * j + 1] - ya, by, iby);
        dz = min_img(g.x[3 * j + 2] - za, bz, ibz);
    };
    auto active = [&](int j) {
        float dx, dy, dz;
        disp(j, dx, dy, dz);
        return dx * dx + dy * dy + dz * dz < cut2;
    };
    auto edge = [&](int j) {
        float dx, dy, dz;
        disp(j, dx, dy, dz);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const int sj = g.species[j];
        if (r2 < rep2 && !is_bonded(g.bonds, a, j)) {
            const float r = sqrtf(r2);
            float dE;
            const float E = rep_pair(g.rep, sa, sj, r, &dE);
            const float c = dE / r;
            fx += c * dx; fy += c * dy; fz += c * dz;
            e += 0.5f * E;
        }
        if (sa == 0 || sj == 0 || g.mol_id[j] == ma || !(r2 < rc2)) return;
        const float r = sqrtf(r2);
        const float sr2 = s2 / r2, sr6 = sr2 * sr2 * sr2;
        const float elj = 4.f * g.lj_eps * (sr6 * sr6 - sr6);
        const float delj = 4.f * g.lj_eps * (-12.f * sr6 * sr6 + 6.f * sr6) / r;
        float du;
        const float fc = envelope(r * inv_rc, g.lj_p, &du);
        const float dE = delj * fc + elj * du * inv_rc;     // dE/dr
        const float c = dE / r;                             // F_a = E'(r) d / r
        fx += c * dx; fy += c * dy; fz += c * dz;
        e += 0.5f * elj * fc;
    };
    for_active_canonical(g.col, g.row_ptr[a], g.row_ptr[a + 1], sh_queue[warp], lane, active, edge);
    if (g.bonds.ptr) bond_force(g.bonds, g.x, a, bx, by, bz, ibx, iby, ibz, lane, fx, fy, fz, e);
    fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz); e = warp_sum(e);
    if (lane == 0) {
        g.F[3 * a] += fx; g.F[3 * a + 1] += fy; g.F[3 * a + 2] += fz;
        if (g.e_atom) g.e_atom[a] += e;
    }
}

void launch_prior(const PriorArgs &a, cudaStream_t st) {
    if (a.n_atoms == 0) return;
    k_prior<<<(a.n_atoms + 3) / 4, 128, 0, st>>>(a);
}

// ----------------------------------------------------------- integrator
// One thread per atom; the operations selected by `ops` run in this order:
// closing B, closing outer kick, opening outer kick, then B-A-O-A.
__global__ void k_integrate(IntegArgs g) {
    if (*g.err) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_atoms) return;
    const float am = kAccConv / g.masses[i];
    float vx = g.v[3 * i], vy = g.v[3 * i + 1], vz = g.v[3 * i + 2];
    const float sfx = g.f_fast[3 * i], sfy = g.f_fast[3 * i + 1], sfz = g.f_fast[3 * i + 2];
    if (g.ops & OP_CLOSE_B) {
        const float h = g.h_in * am;
        vx = fmaf(h, sfx, vx); vy = fmaf(h, sfy, vy); vz = fmaf(h, sfz, vz);
    }
    if (g.ops & (OP_KICK_L | OP_KICK_L2)) {
        const float h = g.h_out * am;
        const float lx = g.f_slow[3 * i] - sfx, ly = g.f_slow[3 * i + 1] - sfy, lz = g.f_slow[3 * i + 2] - sfz;
        if (g.ops & OP_KICK_L) { vx = fmaf(h, lx, vx); vy = fmaf(h, ly, vy); vz = fmaf(h, lz, vz); }
        if (g.ops & OP_KICK_L2) { vx = fmaf(h, lx, vx); vy = fmaf(h, ly, vy); vz = fmaf(h, lz, vz); }
    }
    if (g.ops & OP_BAOA) {
        const float h = g.h_in * am;
        vx = fmaf(h, sfx, vx); vy = fmaf(h, sfy, vy); vz = fmaf(h, sfz, vz);
        float x = g.x[3 * i], y = g.x[3 * i + 1], z = g.x[3 * i + 2];
        x = fmaf(g.h_in, vx, x); y = fmaf(g.h_in, vy, y); z = fmaf(g.h_in, vz, z);
        const int r = g.atom_rep[i];
        const int local = i - g.rep_off[r];
        const float3 G = gauss3(g.seed[r], g.rep_id[r], g.step[r] + g.step_add, (uint32_t)local);
        const int sp = g.species[i];
        const float c1 = g.c1[sp], c2 = g.c2[sp] / sqrtf(g.masses[i]);
        vx = fmaf(c1, vx, c2 * G.x); vy = fmaf(c1, vy, c2 * G.y); vz = fmaf(c1, vz, c2 * G.z);
        x = fmaf(g.h_in, vx, x); y = fmaf(g.h_in, vy, y); z = fmaf(g.h_in, vz, z);
        if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(vx) && isfinite(vy) && isfinite(vz)))
            set_error(g.err, DMTS_E_NONFINITE);
        g.x[3 * i] = x; g.x[3 * i + 1] = y; g.x[3 * i + 2] = z;
        if (g.x_ref) {
            const float ex = x - g.x_ref[3 * i], ey = y - g.x_ref[3 * i + 1], ez = z - g.x_ref[3 * i + 2];
            if (ex * ex + ey * ey + ez * ez > g.half_skin2) *g.rebuild = 1;
        }
    }
    g.v[3 * i] = vx; g.v[3 * i + 1] = vy; g.v[3 * i + 2] = vz;
}

void launch_integrate(const IntegArgs &a, cudaStream_t st) {
    if (a.n_atoms == 0) return;
    k_integrate<<<(a.n_atoms + 255) / 256, 256, 0, st>>>(a);
}

__global__ void k_advance(uint64_t *step, int n_rep, uint64_t add, const int *err) {
    if (*err) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n_rep) step[r] += add;
}

void launch_advance_step(uint64_t *step, int n_rep, uint64_t add, const int *err, cudaStream_t st) {
    if (n_rep == 0) return;
    k_advance<<<(n_rep + 127) / 128, 128, 0, st>>>(step, n_rep, add, err);
}

}  // namespace dmts
