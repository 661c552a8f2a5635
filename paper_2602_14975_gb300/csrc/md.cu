// NC direct-force head (Sec. 2 "Model architecture"), the bonded + LJ prior,
// and the fused BAOAB/RESPA integrator with Philox4x32-10 noise (Algorithm 1);
// the replica-local mean subtraction of the fast force; the virial estimator
// and the piston kernels of the NPT path (Sec. 2, virial term in NPT); and
// the adjoint of the fast force with respect to its weights (head, weight
// contractions, layer gradients) with the Adam update, for distillation of
// the NC model (Sec. 2, "Model training").
#include <algorithm>
#include "md.cuh"
#include "mp.cuh"
#include "ptx.cuh"

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
    count_launch();
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
    count_launch();
}

// Bond entry q of atom a (d = x_j - x_a): the force on a, k (r - r0) d / r,
// its energy and pair-form virial. The same bond seen from j gives exactly
// the opposite force (d exactly negated, the same r and factor).
// Harmonic bond term of atom a with its partner at (xj, yj, zj), rest length r0.
__device__ __forceinline__ void bond_term_at(float k, float xj, float yj, float zj, float r0, float xa, float ya,
                                             float za, float bx, float by, float bz, float ibx, float iby, float ibz,
                                             float &gx, float &gy, float &gz, float &e, float &w) {
    const float dx = min_img(xj - xa, bx, ibx);
    const float dy = min_img(yj - ya, by, iby);
    const float dz = min_img(zj - za, bz, ibz);
    const float r = sqrtf(dx * dx + dy * dy + dz * dz);
    const float dr = r - r0;
    const float g = k * dr / r;
    gx = g * dx; gy = g * dy; gz = g * dz;
    e = 0.25f * k * dr * dr;              // each bond is listed by both atoms
    w = 0.5f * g * r * r;                 // pair-form virial, half per listed direction
}

__device__ __forceinline__ void bond_term(const BondTable &b, const float *x, int q, float xa, float ya, float za,
                                          float bx, float by, float bz, float ibx, float iby, float ibz, float &gx,
                                          float &gy, float &gz, float &e, float &w) {
    const int j = b.idx[q];
    bond_term_at(b.k, x[3 * j], x[3 * j + 1], x[3 * j + 2], b.r0[q], xa, ya, za, bx, by, bz, ibx, iby, ibz, gx, gy, gz,
                 e, w);
}

__device__ __forceinline__ void bond_force(const BondTable &b, const float *x, int a, float bx, float by,
                                           float bz, float ibx, float iby, float ibz, int lane, float &fx,
                                           float &fy, float &fz, float &e, float *w = nullptr) {
    const float xa = x[3 * a], ya = x[3 * a + 1], za = x[3 * a + 2];
    for (int q = b.ptr[a] + lane; q < b.ptr[a + 1]; q += 32) {
        float gx, gy, gz, eq, wq;
        bond_term(b, x, q, xa, ya, za, bx, by, bz, ibx, iby, ibz, gx, gy, gz, eq, wq);
        fx += gx; fy += gy; fz += gz;
        e += eq;
        if (w) *w += wq;
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
// Each pair (a, j), a < j, within r_c is evaluated once, by atom a's warp:
//   c_ajh = q_ah . k_jh / sqrt(n_c),  c_jah = q_jh . k_ah / sqrt(n_c)
//   F_aj = (sum_{h<K} c_ajh B_h) (n + sum_{h<n_l} c_aj(K+h) V_ah) f_c
//   F_ja = (sum_{h<K} c_jah B_h) (-n + sum_{h<n_l} c_ja(K+h) V_jh) f_c
//   P_aj = scale (F_aj - F_ja) (+ the screened repulsion of the pair)
// which enters F_a with + and F_j with - (the antisymmetric sum), so every
// pair costs one evaluation instead of one from each end. Forces are summed
// in 32.32 fixed point with 64-bit integer atomics: integer addition is
// exact and associative, so F does not depend on the order in which warps
// add their terms, nor on the skin entries of the list (bit-reproducible
// alone or batched). k_nc_convert converts F to fp32 and clears it.
// Upper active neighbours (j > a) are taken 16 at a time (the g-th in
// batch g / 16 on lanes g % 16 and g % 16 + 16): the first lane of each pair
// bulk-copies the neighbour's q/k row into shared memory, the second loads
// the neighbour's tensor-head vectors (its heads), both evaluate the radial
// part while the row arrives, and each forms the dot products of half of
// the heads. The warps are persistent (one per block, as many blocks as fit)
// and take atoms from a work counter in processing order; each loads its
// next atom's row, candidates and own values one atom ahead (see the kernel).
constexpr int NCH_WARPS = 1;
__device__ __forceinline__ double fix_sum_to_double(unsigned long long s) {
    return (double)(long long)s * (1.0 / 4294967296.0);   // exact for |s| < 2^53
}
// Mean force of replica r from its exact fixed-point sum (FP64, as used by
// the subtraction).
// The sums of the head's forces cancel exactly (every term enters two atoms
// with opposite signs), so a zero sum is the rule and skips the division.
__device__ __forceinline__ float fix_mean1(unsigned long long s, double n) {
    return s == 0ull ? 0.f : (float)(fix_sum_to_double(s) / n);
}
__device__ __forceinline__ float3 fix_mean(const unsigned long long *sum, const int *rep_off, int r) {
    const double n = (double)(rep_off[r + 1] - rep_off[r]);
    return make_float3(fix_mean1(sum[3 * r], n), fix_mean1(sum[3 * r + 1], n), fix_mean1(sum[3 * r + 2], n));
}
// Sum of a 64-bit integer over the lanes whose key equals this lane's (the
// lanes of one replica); every lane takes part.
__device__ __forceinline__ long long seg_sum_ll(long long v, int key) {
    const int k0 = __shfl_sync(DMTS_FULL, key, 0);
    if (__all_sync(DMTS_FULL, key == k0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(DMTS_FULL, v, o);
        return v;
    }
    const unsigned peers = __match_any_sync(DMTS_FULL, key);
    long long t = 0;
    for (int src = 0; src < 32; ++src) {
        const long long u = __shfl_sync(DMTS_FULL, v, src);
        if ((peers >> src) & 1u) t += u;
    }
    return t;
}

template <int K, int NC, int NL>
struct NCHeadSmem {
    static constexpr int H = K + NL, QKW = 2 * H * NC;
    static constexpr int RSTR = QKW + 4;    // padded row stride (floats): conflict-free 16-byte reads
    static constexpr int ROWB = QKW * 4;    // bytes copied per row
    static constexpr int BATCH = 16;        // neighbours per staged batch
    static constexpr int HH = (H + 1) / 2;  // heads per lane of a pair
    static constexpr int VS = nc_v_stride(NL);   // V row stride (floats)
    static constexpr size_t rows = (size_t)NCH_WARPS * BATCH * RSTR * 4;
    static constexpr size_t qk = (size_t)NCH_WARPS * QKW * 4;
    static constexpr size_t vv = (size_t)NCH_WARPS * 4 * NL * 4;
    static constexpr size_t queue = (size_t)NCH_WARPS * 64 * 4;
    static constexpr size_t qdisp = (size_t)NCH_WARPS * 64 * 3 * 4;   // displacement of each queued edge
    static constexpr size_t bytes = rows + qk + vv + queue + qdisp + NCH_WARPS * 8;
    static_assert(QKW % 16 == 0, "row stride");
    static_assert(HH <= K, "each lane's first heads are Bessel heads");
};

template <int K, int NC, int NL>
__global__ void __launch_bounds__(NCH_WARPS * 32) k_nc_head(NCHeadArgs g) {
    using SM = NCHeadSmem<K, NC, NL>;
    constexpr int H = SM::H, QKW = SM::QKW, RSTR = SM::RSTR;
    extern __shared__ __align__(16) unsigned char nch_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int BATCH = SM::BATCH, HH = SM::HH;
    float *rows = reinterpret_cast<float *>(nch_smem) + (size_t)warp * BATCH * RSTR;
    unsigned char *rest = nch_smem + SM::rows;
    float *qa = reinterpret_cast<float *>(rest) + warp * QKW;
    float *va = reinterpret_cast<float *>(rest + SM::qk) + warp * 4 * NL;
    int *queue = reinterpret_cast<int *>(rest + SM::qk + SM::vv) + warp * 64;
    float *qd = reinterpret_cast<float *>(rest + SM::qk + SM::vv + SM::queue) + warp * 64 * 3;
    uint64_t *bar_p = reinterpret_cast<uint64_t *>(rest + SM::qk + SM::vv + SM::queue + SM::qdisp) + warp;
    const uint32_t bar = smem_u32(bar_p);
    // the per-replica sums of the last evaluation have been consumed: clear
    // them for this one's conversion
    if (blockIdx.x == 0 && g.sum)
        for (int t = threadIdx.x; t < 3 * g.n_rep; t += blockDim.x) g.sum[t] = 0ull;
    if (*g.err) return;
    // The warps take atoms from a counter, in processing order, as they free
    // up. A warp's first atom's row and first 32 candidates are loaded here,
    // every later atom's one atom ahead, in stages behind the current atom's
    // work: the counter at its start, the atom index before its last batch,
    // the row bounds after it, the candidates after its bonds and their
    // positions after its force sums.
    int wa = __shfl_sync(DMTS_FULL, lane == 0 ? (int)atomicAdd(g.next, 1u) : 0, 0);
    if (wa >= g.n_atoms) return;
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    __syncwarp();
    uint32_t phase = 0;
    constexpr int QR = (QKW + 31) / 32;   // q/k row values per lane
    const bool with_rep = g.bonds.ptr && g.rep.on;
    int a = g.order ? __ldg(g.order + wa) : wa;
    int beg = g.row_ptr[a], end = g.row_ptr[a + 1];
    int cj = beg + lane < end ? __ldg(g.col + beg + lane) : -1;
    float cx = 0.f, cy = 0.f, cz = 0.f;
    if (cj >= 0) {
        cx = __ldg(g.x + 3 * cj);
        cy = __ldg(g.x + 3 * cj + 1);
        cz = __ldg(g.x + 3 * cj + 2);
    }
    // the atom's own values: its q/k row and tensor-head vectors (one share
    // per lane), position, replica box, species, and its bonds (lane q holds
    // bond q: partner index, position and rest length)
    float qr[QR], vr = 0.f;
#pragma unroll
    for (int u = 0; u < QR; ++u) qr[u] = lane + 32 * u < QKW ? g.QK[(size_t)a * QKW + lane + 32 * u] : 0.f;
    if (lane < NL * 3) vr = g.V[(size_t)a * SM::VS + lane];
    int rep = g.atom_rep[a], sa = g.species[a];
    float xa = g.x[3 * a], ya = g.x[3 * a + 1], za = g.x[3 * a + 2];
    float bx = g.box[3 * rep], by = g.box[3 * rep + 1], bz = g.box[3 * rep + 2];
    int q0 = 0, nbond = 0, jb = -1;
    float bjx = 0.f, bjy = 0.f, bjz = 0.f, br0 = 0.f;
    if (g.bonds.ptr) {
        q0 = g.bonds.ptr[a];
        nbond = g.bonds.ptr[a + 1] - q0;
        if (lane < nbond) {
            jb = __ldg(g.bonds.idx + q0 + lane);
            bjx = __ldg(g.x + 3 * jb);
            bjy = __ldg(g.x + 3 * jb + 1);
            bjz = __ldg(g.x + 3 * jb + 2);
            br0 = __ldg(g.bonds.r0 + q0 + lane);
        }
    }
    for (;;) {
        const int wn_raw = lane == 0 ? (int)atomicAdd(g.next, 1u) : 0;   // read after the candidates
        int wn = 0, an = 0, bn = 0, en = 0, cjn = -1;
        bool more = false;
        // the next atom's own values, loaded in the same stages as its row
        float qrn[QR], vrn = 0.f;
        int repn = 0, san = 0, q0n = 0, nbondn = 0, jbn = -1;
        float xan = 0.f, yan = 0.f, zan = 0.f, bxn = 0.f, byn = 0.f, bzn = 0.f;
#pragma unroll
        for (int u = 0; u < QR; ++u)
            if (lane + 32 * u < QKW) qa[lane + 32 * u] = qr[u];
        if (lane < NL * 3) va[lane] = vr;
        __syncwarp();
        const float *ka = qa + H * NC;
        const float ibx = bx > 0.f ? 1.f / bx : 0.f, iby = by > 0.f ? 1.f / by : 0.f, ibz = bz > 0.f ? 1.f / bz : 0.f;
        const float rc2 = g.rc * g.rc, isnc = rsqrtf((float)NC);
        const float rep2 = g.rep.rc * g.rep.rc;
        // bonded partners of a (up to four, from the lanes holding its bonds;
        // more fall back to the table)
        int bp[4] = {-1, -1, -1, -1};
        const int nbp = with_rep ? nbond : 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = __shfl_sync(DMTS_FULL, jb, q);
            if (q < nbp) bp[q] = t;
        }
        auto bonded = [&](int j) {
            if (nbp > 4) return is_bonded(g.bonds, a, j);
            return j == bp[0] || j == bp[1] || j == bp[2] || j == bp[3];
        };
        long long ox = 0, oy = 0, oz = 0;     // this lane's share of a's side of its pairs, fixed point
        float wv = 0.f;                       // virial proxy: (F_aj - F_ja) . d_aj (+ repulsion) over a's pairs
        bool bad = false;                     // a pair term outside the fixed-point range (or not finite)
        bool alive = true;

        // one batch: lanes e and e + 16 (e < nb) own queued edge taken + e; the
        // first stages the row and adds the repulsion, the pair splits the heads
        const int slot = lane & (BATCH - 1), half = lane / BATCH;
        auto batch = [&](int taken, int nb) {
            const int qs = (taken + slot) & 63;
            const int j = slot < nb ? queue[qs] : -1;
            fence_proxy_async_smem();      // earlier reads of the rows before the copies overwrite them
            if (lane == 0) mbar_expect_tx(bar, (uint32_t)nb * SM::ROWB);
            __syncwarp();
            if (j >= 0 && half == 0) bulk_g2s(smem_u32(rows + slot * RSTR), g.QK + (size_t)j * QKW, SM::ROWB, bar);
            // the neighbour's tensor-head vectors, for the lane of the pair that
            // owns the tensor heads (plain loads: 12 bytes per head)
            float vj[3 * NL];
#pragma unroll
            for (int q = 0; q < 3 * NL; ++q) vj[q] = (j >= 0 && half == 1) ? __ldg(g.V + (size_t)j * SM::VS + q) : 0.f;
            // radial part of the edge while the rows arrive
            float dx = 0.f, dy = 0.f, dz = 0.f, inv = 1.f, fc = 0.f, Bh[HH], crep = 0.f, r2 = 0.f;
            if (j >= 0) {
                dx = qd[3 * qs];
                dy = qd[3 * qs + 1];
                dz = qd[3 * qs + 2];
                r2 = dx * dx + dy * dy + dz * dz;
                const float r = sqrtf(r2);
                inv = 1.f / r;
                if (half == 0 && with_rep && r2 < rep2 && !bonded(j)) {
                    float dE;
                    rep_pair(g.rep, sa, g.species[j], r, &dE);
                    crep = dE * inv;               // F_a = E'(r) d / r, F_j = -F_a
                }
                float du;
                fc = envelope(r * g.inv_rc, g.p, &du);
                float B[K];
                bessel<K, false>(r, g.inv_rc, g.bnorm, B, nullptr);
#pragma unroll
                for (int hl = 0; hl < HH; ++hl)
                    Bh[hl] = half == 0 ? B[hl] : (HH + hl < K ? B[HH + hl < K ? HH + hl : 0] : 0.f);
            }
            const bool got = __all_sync(DMTS_FULL, mbar_wait(bar, phase));
            phase ^= 1u;
            if (!got) {
                // record the timeout, give the copies in flight a last bounded
                // wait, and stop
                if (lane == 0) atomicCAS(g.err, 0, (int)DMTS_E_TIMEOUT);
                mbar_wait(bar, phase ^ 1u);
                alive = false;
                return;
            }
            // partial sums over this lane's heads h = half * HH + hl
            float part[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // Saj, Sja, va (3), vj (3)
            if (j >= 0) {
                const float *row = rows + slot * RSTR;
#pragma unroll
                for (int hl = 0; hl < HH; ++hl) {
                    const int h = half * HH + hl;
                    if (h < H) {
                        const float4 *qj4 = reinterpret_cast<const float4 *>(row + h * NC);
                        const float4 *kj4 = reinterpret_cast<const float4 *>(row + (H + h) * NC);
                        const float4 *qa4 = reinterpret_cast<const float4 *>(qa + h * NC);
                        const float4 *ka4 = reinterpret_cast<const float4 *>(ka + h * NC);
                        float caj = 0.f, cja = 0.f;
#pragma unroll
                        for (int q = 0; q < NC / 4; ++q) {
                            const float4 kj = kj4[q], qj = qj4[q], qi = qa4[q], ki = ka4[q];
                            caj = fmaf(qi.x, kj.x, fmaf(qi.y, kj.y, fmaf(qi.z, kj.z, fmaf(qi.w, kj.w, caj))));
                            cja = fmaf(qj.x, ki.x, fmaf(qj.y, ki.y, fmaf(qj.z, ki.z, fmaf(qj.w, ki.w, cja))));
                        }
                        caj *= isnc;
                        cja *= isnc;
                        if (h < K) {
                            part[0] = fmaf(caj, Bh[hl], part[0]);
                            part[1] = fmaf(cja, Bh[hl], part[1]);
                        } else {
                            // tensor heads lie in the second lane's half (HH <= K): t is static
                            const int t = HH + hl - K;
#pragma unroll
                            for (int cmp = 0; cmp < 3; ++cmp) {
                                part[2 + cmp] = fmaf(caj, va[3 * t + cmp], part[2 + cmp]);
                                part[5 + cmp] = fmaf(cja, vj[3 * t + cmp], part[5 + cmp]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) part[q] += __shfl_xor_sync(DMTS_FULL, part[q], BATCH);
            if (j >= 0 && half == 0) {
                const float nx = dx * inv, ny = dy * inv, nz = dz * inv;
                const float pa = part[0] * fc, pj = part[1] * fc;
                const float ux = pa * (nx + part[2]) - pj * (-nx + part[5]);
                const float uy = pa * (ny + part[3]) - pj * (-ny + part[6]);
                const float uz = pa * (nz + part[4]) - pj * (-nz + part[7]);
                const float px = fmaf(g.scale, ux, crep * dx), py = fmaf(g.scale, uy, crep * dy),
                            pz = fmaf(g.scale, uz, crep * dz);
                wv += fmaf(g.scale, ux * dx + uy * dy + uz * dz, crep * r2);
                if (fabsf(px) < kFixMax && fabsf(py) < kFixMax && fabsf(pz) < kFixMax) {
                    const long long qx = to_fix(px), qy = to_fix(py), qz = to_fix(pz);
                    ox += qx; oy += qy; oz += qz;
                    unsigned long long *fj = g.Ffix + 3 * (size_t)j;
                    fix_add(fj, -qx); fix_add(fj + 1, -qy); fix_add(fj + 2, -qz);
                } else {
                    bad = true;   // not finite, or a blow-up beyond the fixed-point range
                }
            }
            __syncwarp();
        };

        int queued = 0, taken = 0;
        for (int base = beg; base < end && alive; base += 32) {
            const int e = base + lane;
            const bool first = base == beg;   // prefetched
            const int j = first ? cj : (e < end ? __ldg(g.col + e) : -1);
            bool act = false;
            float dx = 0.f, dy = 0.f, dz = 0.f;
            if (j > a) {
                dx = min_img((first ? cx : __ldg(g.x + 3 * j)) - xa, bx, ibx);
                dy = min_img((first ? cy : __ldg(g.x + 3 * j + 1)) - ya, by, iby);
                dz = min_img((first ? cz : __ldg(g.x + 3 * j + 2)) - za, bz, ibz);
                act = dx * dx + dy * dy + dz * dz < rc2;
            }
            const unsigned m = __ballot_sync(DMTS_FULL, act);
            if (act) {
                const int qs = (queued + __popc(m & ((1u << lane) - 1u))) & 63;
                queue[qs] = j;
                qd[3 * qs] = dx;
                qd[3 * qs + 1] = dy;
                qd[3 * qs + 2] = dz;
            }
            queued += __popc(m);
            __syncwarp();
            while (queued - taken >= BATCH && alive) {
                batch(taken, BATCH);
                taken += BATCH;
            }
        }
        // the next atom
        wn = __shfl_sync(DMTS_FULL, wn_raw, 0);
        more = wn < g.n_atoms;
        if (more) an = g.order ? __ldg(g.order + wn) : wn;
        if (alive && queued > taken) batch(taken, queued - taken);
        if (!alive) return;
        if (more) {   // its row bounds and own values
            bn = g.row_ptr[an];
            en = g.row_ptr[an + 1];
#pragma unroll
            for (int u = 0; u < QR; ++u) qrn[u] = lane + 32 * u < QKW ? g.QK[(size_t)an * QKW + lane + 32 * u] : 0.f;
            if (lane < NL * 3) vrn = g.V[(size_t)an * SM::VS + lane];
            repn = g.atom_rep[an];
            san = g.species[an];
            xan = g.x[3 * an];
            yan = g.x[3 * an + 1];
            zan = g.x[3 * an + 2];
            if (g.bonds.ptr) {
                q0n = g.bonds.ptr[an];
                nbondn = g.bonds.ptr[an + 1] - q0n;
            }
        }
        float w = wv;
        if (g.bonds.ptr) {
            // bonds in fixed point too: the two ends' terms cancel exactly
            for (int q = lane; q < nbond; q += 32) {
                float gx, gy, gz, eq, wq;
                if (q < 32)   // the prefetched bond of this lane
                    bond_term_at(g.bonds.k, bjx, bjy, bjz, br0, xa, ya, za, bx, by, bz, ibx, iby, ibz, gx, gy, gz, eq,
                                 wq);
                else
                    bond_term(g.bonds, g.x, g.bonds.ptr[a] + q, xa, ya, za, bx, by, bz, ibx, iby, ibz, gx, gy, gz, eq,
                              wq);
                if (fabsf(gx) < kFixMax && fabsf(gy) < kFixMax && fabsf(gz) < kFixMax) {
                    ox += to_fix(gx); oy += to_fix(gy); oz += to_fix(gz);
                } else {
                    bad = true;
                }
                w += wq;
            }
        }
        if (bn + lane < en) cjn = __ldg(g.col + bn + lane);   // its first candidates, box and bond partners
        if (more) {
            bxn = g.box[3 * repn];
            byn = g.box[3 * repn + 1];
            bzn = g.box[3 * repn + 2];
            if (lane < nbondn) jbn = __ldg(g.bonds.idx + q0n + lane);
        }
        if (__any_sync(DMTS_FULL, bad)) {
            if (lane == 0) set_error(g.err, DMTS_E_NONFINITE);
            return;
        }
        ox = seg_sum_ll(ox, 0); oy = seg_sum_ll(oy, 0); oz = seg_sum_ll(oz, 0);
        if (g.W) w = warp_sum(w);
        if (lane == 0) {
            unsigned long long *fa = g.Ffix + 3 * (size_t)a;
            fix_add(fa, ox); fix_add(fa + 1, oy); fix_add(fa + 2, oz);
            if (g.W) g.W[a] = w;
        }
        if (!more) break;
        float cxn = 0.f, cyn = 0.f, czn = 0.f, bjxn = 0.f, bjyn = 0.f, bjzn = 0.f, br0n = 0.f;
        if (cjn >= 0) {
            cxn = __ldg(g.x + 3 * cjn);
            cyn = __ldg(g.x + 3 * cjn + 1);
            czn = __ldg(g.x + 3 * cjn + 2);
        }
        if (jbn >= 0) {
            bjxn = __ldg(g.x + 3 * jbn);
            bjyn = __ldg(g.x + 3 * jbn + 1);
            bjzn = __ldg(g.x + 3 * jbn + 2);
            br0n = __ldg(g.bonds.r0 + q0n + lane);
        }
        wa = wn;
        a = an;
        beg = bn;
        end = en;
        cj = cjn;
        cx = cxn;
        cy = cyn;
        cz = czn;
#pragma unroll
        for (int u = 0; u < QR; ++u) qr[u] = qrn[u];
        vr = vrn;
        rep = repn;
        sa = san;
        xa = xan;
        ya = yan;
        za = zan;
        bx = bxn;
        by = byn;
        bz = bzn;
        nbond = nbondn;
        jb = jbn;
        bjx = bjxn;
        bjy = bjyn;
        bjz = bjzn;
        br0 = br0n;
        __syncwarp();   // this atom's reads of qa, va and the queue are done
    }
}

template <int K, int NC, int NL>
static void nc_head_launch(const NCHeadArgs &a, cudaStream_t st) {
    using SM = NCHeadSmem<K, NC, NL>;
    // per launch: the attribute belongs to the current device's context
    cudaFuncSetAttribute(k_nc_head<K, NC, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
    // persistent: as many warps as fit on the GPU at once, each taking every
    // (grid)-th atom
    static int resident = 0;
    if (!resident) {
        int dev = 0, n_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        resident = std::max(1, n_sm * resident_ctas(reinterpret_cast<const void *>(k_nc_head<K, NC, NL>),
                                                    NCH_WARPS * 32, SM::bytes, dev));
    }
    const int blocks = std::min((a.n_atoms + NCH_WARPS - 1) / NCH_WARPS, resident);
    k_nc_head<K, NC, NL><<<blocks, NCH_WARPS * 32, SM::bytes, st>>>(a);
    count_launch();
}

void launch_nc_head(int K, int n_c, int n_l, const NCHeadArgs &a, cudaStream_t st) {
    if (a.n_atoms == 0) return;
    if (K == 8 && n_c == 8 && n_l == 2) nc_head_launch<8, 8, 2>(a, st);
    else if (K == 8 && n_c == 8 && n_l == 1) nc_head_launch<8, 8, 1>(a, st);
    else if (K == 8 && n_c == 8 && n_l == 3) nc_head_launch<8, 8, 3>(a, st);
    else if (K == 8 && n_c == 8 && n_l == 4) nc_head_launch<8, 8, 4>(a, st);
}

// ------------------------------------------------- NC head adjoint (q/k)
// Warp per atom a. Lane h < H owns head h of c_ajh = q_ah . k_jh / sqrt(n_c)
// (and accumulates dL/dq_ah), lane H + h owns c_jah = q_jh . k_ah / sqrt(n_c)
// (dL/dk_ah). With F_aj = f_c S_aj (n + T_aj), S_aj = sum_{h<K} c_ajh B_h,
// T_aj = sum_t c_aj(K+t) V_at, F_ja = f_c S_ja (-n + T_ja) and
// F_a = scale sum_j (F_aj - F_ja) (+ terms without q/k), each directed pair
// enters F_a with + and F_j with -, so u = scale (gF_a - gF_j) and
//   dL/dc_ajh = f_c B_h u.(n + T_aj)   (h < K),  f_c S_aj u.V_at  (h = K + t),
//   dL/dc_jah = -f_c B_h u.(-n + T_ja) (h < K), -f_c S_ja u.V_jt  (h = K + t).
// Each pair is visited from both ends, so every atom gathers its own rows'
// gradients: no atomics, deterministic.
template <int K, int NC, int NL>
__global__ void __launch_bounds__(128) k_nc_head_bwd(NCHeadArgs g, const float *__restrict__ gF,
                                                    float *__restrict__ gQK, float *__restrict__ gV) {
    constexpr int H = K + NL, QKW = 2 * H * NC;
    static_assert(2 * H <= 32, "one lane per head and role");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wa = blockIdx.x * 4 + warp;
    if (wa >= g.n_atoms || *g.err) return;
    const int a = g.order ? __ldg(g.order + wa) : wa;
    const bool role_aj = lane < H, live = lane < 2 * H;
    const int h = role_aj ? lane : (live ? lane - H : 0);
    const float isnc = rsqrtf((float)NC);
    // own row: q_a[h] (role aj) or k_a[h] (role ja)
    float mine[NC], acc[NC], accv[3] = {0.f, 0.f, 0.f};   // accv: dL/dV_at on the tensor-head lanes of role aj
    const float *ra = g.QK + (size_t)a * QKW + (role_aj ? 0 : H * NC) + h * NC;
#pragma unroll
    for (int d = 0; d < NC; ++d) {
        mine[d] = live ? ra[d] : 0.f;
        acc[d] = 0.f;
    }
    float va[3 * NL];
#pragma unroll
    for (int t = 0; t < 3 * NL; ++t) va[t] = g.V[(size_t)a * nc_v_stride(NL) + t];
    const float gax = gF[3 * a], gay = gF[3 * a + 1], gaz = gF[3 * a + 2];
    const int rep = g.atom_rep[a];
    const float bx = g.box[3 * rep], by = g.box[3 * rep + 1], bz = g.box[3 * rep + 2];
    const float ibx = bx > 0.f ? 1.f / bx : 0.f, iby = by > 0.f ? 1.f / by : 0.f, ibz = bz > 0.f ? 1.f / bz : 0.f;
    const float xa = g.x[3 * a], ya = g.x[3 * a + 1], za = g.x[3 * a + 2];
    const float rc2 = g.rc * g.rc;
    for (int e = g.row_ptr[a]; e < g.row_ptr[a + 1]; ++e) {
        const int j = __ldg(g.col + e);
        const float dx = min_img(__ldg(g.x + 3 * j) - xa, bx, ibx);
        const float dy = min_img(__ldg(g.x + 3 * j + 1) - ya, by, iby);
        const float dz = min_img(__ldg(g.x + 3 * j + 2) - za, bz, ibz);
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < rc2)) continue;   // uniform over the warp
        const float r = sqrtf(r2), inv = 1.f / r;
        const float nx = dx * inv, ny = dy * inv, nz = dz * inv;
        float du;
        const float fc = envelope(r * g.inv_rc, g.p, &du);
        float B[K];
        bessel<K, false>(r, g.inv_rc, g.bnorm, B, nullptr);
        float Bh = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) Bh = (h == k) ? B[k] : Bh;
        // the other atom's row: k_j[h] (role aj) or q_j[h] (role ja)
        float other[NC];
        const float *rj = g.QK + (size_t)j * QKW + (role_aj ? H * NC : 0) + h * NC;
        float c = 0.f;
#pragma unroll
        for (int d = 0; d < NC; ++d) {
            other[d] = live ? __ldg(rj + d) : 0.f;
            c = fmaf(mine[d], other[d], c);
        }
        c *= isnc;
        const bool bes = live && h < K;
        const int t = h - K;
        float vt[3] = {0.f, 0.f, 0.f};   // V_at (role aj) or V_jt (role ja) of this tensor head
        if (live && h >= K) {
#pragma unroll
            for (int q = 0; q < 3; ++q)
                vt[q] = role_aj ? va[3 * (t < NL ? t : 0) + q]
                                : __ldg(g.V + (size_t)j * nc_v_stride(NL) + 3 * (t < NL ? t : 0) + q);
        }
        const float sB = bes ? c * Bh : 0.f;
        const float S_aj = warp_sum(role_aj ? sB : 0.f), S_ja = warp_sum(role_aj ? 0.f : sB);
        float T_aj[3], T_ja[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float cv = (live && h >= K) ? c * vt[q] : 0.f;
            T_aj[q] = warp_sum(role_aj ? cv : 0.f);
            T_ja[q] = warp_sum(role_aj ? 0.f : cv);
        }
        const float ux = g.scale * (gax - __ldg(gF + 3 * j)), uy = g.scale * (gay - __ldg(gF + 3 * j + 1)),
                    uz = g.scale * (gaz - __ldg(gF + 3 * j + 2));
        float G;
        if (role_aj) {
            G = h < K ? fc * Bh * (ux * (nx + T_aj[0]) + uy * (ny + T_aj[1]) + uz * (nz + T_aj[2]))
                      : fc * S_aj * (ux * vt[0] + uy * vt[1] + uz * vt[2]);
        } else {
            G = h < K ? -fc * Bh * (ux * (-nx + T_ja[0]) + uy * (-ny + T_ja[1]) + uz * (-nz + T_ja[2]))
                      : -fc * S_ja * (ux * vt[0] + uy * vt[1] + uz * vt[2]);
        }
        if (role_aj && h >= K) {
            // V_at enters F_aj = f_c S_aj (n + sum_t c_aj(K+t) V_at) only
            const float f = fc * S_aj * c;
            accv[0] = fmaf(f, ux, accv[0]); accv[1] = fmaf(f, uy, accv[1]); accv[2] = fmaf(f, uz, accv[2]);
        }
        G *= isnc;
#pragma unroll
        for (int d = 0; d < NC; ++d) acc[d] = fmaf(G, other[d], acc[d]);
    }
    if (gV && role_aj && h >= K) {
        float *o = gV + ((size_t)a * NL + (h - K)) * 3;
        o[0] = accv[0]; o[1] = accv[1]; o[2] = accv[2];
    }
    if (live) {
        const int c0 = (role_aj ? 0 : H * NC) + h * NC;
#pragma unroll
        for (int d = 0; d < NC; ++d) gQK[(size_t)a * QKW + c0 + d] = acc[d];
    }
}

template <int K, int NC, int NL>
static void nc_head_bwd_launch(const NCHeadArgs &a, const float *gF, float *gQK, float *gV, cudaStream_t st) {
    k_nc_head_bwd<K, NC, NL><<<(a.n_atoms + 3) / 4, 128, 0, st>>>(a, gF, gQK, gV);
    count_launch();
}

void launch_nc_head_bwd(int K, int n_c, int n_l, const NCHeadArgs &a, const float *gF, float *gQK, float *gV,
                        cudaStream_t st) {
    if (a.n_atoms == 0) return;
    if (K == 8 && n_c == 8 && n_l == 2) nc_head_bwd_launch<8, 8, 2>(a, gF, gQK, gV, st);
    else if (K == 8 && n_c == 8 && n_l == 1) nc_head_bwd_launch<8, 8, 1>(a, gF, gQK, gV, st);
    else if (K == 8 && n_c == 8 && n_l == 3) nc_head_bwd_launch<8, 8, 3>(a, gF, gQK, gV, st);
    else if (K == 8 && n_c == 8 && n_l == 4) nc_head_bwd_launch<8, 8, 4>(a, gF, gQK, gV, st);
}

// ------------------------------------------------ weight gradients (A^T B)
// Block (32 x 8 threads) = a 32 x 32 output tile over one slice of atoms;
// thread (ty, tx) sums outputs (ty + 8k, tx), k < 4, in atom order.
constexpr int ATB_T = 32, ATB_CH = 16, ATB_SLICES = 64;

__global__ void __launch_bounds__(256) k_atb_part(int N, int O, int I, const float *__restrict__ G,
                                                 const float *__restrict__ X, float *__restrict__ part, int with_cs,
                                                 int slices) {
    __shared__ float Gs[ATB_CH][ATB_T], Xs[ATB_CH][ATB_T];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int o0 = blockIdx.x * ATB_T, i0 = blockIdx.y * ATB_T, sl = blockIdx.z;
    const int per = (N + slices - 1) / slices, a0 = sl * per, a1 = min(N, a0 + per);
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, cs[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c0 = a0; c0 < a1; c0 += ATB_CH) {
        for (int q = threadIdx.x; q < ATB_CH * ATB_T; q += 256) {
            const int aa = q / ATB_T, cc = q % ATB_T, at = c0 + aa;
            Gs[aa][cc] = (at < a1 && o0 + cc < O) ? G[(size_t)at * O + o0 + cc] : 0.f;
            Xs[aa][cc] = (at < a1 && i0 + cc < I) ? X[(size_t)at * I + i0 + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int aa = 0; aa < ATB_CH; ++aa) {
            const float xv = Xs[aa][tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                acc[k] = fmaf(Gs[aa][ty + 8 * k], xv, acc[k]);
                cs[k] += Gs[aa][ty + 8 * k];
            }
        }
        __syncthreads();
    }
    float *pp = part + (size_t)sl * O * (I + 1);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int o = o0 + ty + 8 * k, i = i0 + tx;
        if (o < O && i < I) pp[(size_t)o * (I + 1) + i] = acc[k];
        if (with_cs && o < O && blockIdx.y == 0 && tx == 0) pp[(size_t)o * (I + 1) + I] = cs[k];
    }
}

__global__ void k_atb_reduce(int O, int I, const float *__restrict__ part, float *__restrict__ out,
                             float *__restrict__ cs, int slices) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= O * (I + 1)) return;
    const int o = q / (I + 1), i = q % (I + 1);
    if (i == I && !cs) return;
    float t = 0.f;
    for (int s = 0; s < slices; ++s) t += part[(size_t)s * O * (I + 1) + q];
    if (i < I) out[(size_t)o * I + i] = t;
    else cs[o] = t;
}

void launch_atb(int N, int O, int I, const float *G, const float *X, float *out, float *cs, float *part,
                cudaStream_t st) {
    if (O == 0 || I == 0) return;
    const int slices = std::max(1, std::min(ATB_SLICES, (N + 255) / 256));
    dim3 grid((O + ATB_T - 1) / ATB_T, (I + ATB_T - 1) / ATB_T, slices);
    k_atb_part<<<grid, 256, 0, st>>>(N, O, I, G, X, part, cs != nullptr, slices);
    count_launch();
    const int tot = O * (I + 1);
    k_atb_reduce<<<(tot + 255) / 256, 256, 0, st>>>(O, I, part, out, cs, slices);
    count_launch();
}

// ------------------------------------------- NC layer weight gradients
// Blocks of four warps take atoms in a grid stride; lanes own channel sets
// (C / 32 each); every lane sweeps the atom's active edges in list order.
// Each block adds its warps' sums in warp order into its partial row, and
// k_sum_rows adds the blocks' rows in block order: deterministic.
constexpr int WG_BLOCKS = 1024;

template <int C>
__global__ void __launch_bounds__(128) k_nc_layer_wgrad(NCLayerGradArgs g, float *__restrict__ part) {
    constexpr int K = 8, CPW = C / 32, NW = 2 * K * C;
    __shared__ float red[4][NW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float wacc[2][K][CPW];
#pragma unroll
    for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int u = 0; u < CPW; ++u) wacc[l][k][u] = 0.f;
    const float rc2 = g.rc * g.rc;
    for (int i = blockIdx.x * 4 + warp; i < g.n_atoms && !*g.err; i += gridDim.x * 4) {
        float gA[4][CPW];
#pragma unroll
        for (int u = 0; u < CPW; ++u) {
            const int c = lane * CPW + u;
            const float g0 = g.gq[(size_t)i * 2 * C + c], g1 = g.gq[(size_t)i * 2 * C + C + c];
            gA[0][u] = 2.f * g.A[((size_t)i * 4) * C + c] * g0;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                float t = 2.f * g.A[((size_t)i * 4 + 1 + m) * C + c] * g1;
                for (int h = 0; h < g.n_l; ++h) t = fmaf(g.U[h * C + c], g.gV[((size_t)i * g.n_l + h) * 3 + m], t);
                gA[1 + m][u] = t;
            }
        }
        const int rep = g.atom_rep[i];
        const float bx = g.box[3 * rep], by = g.box[3 * rep + 1], bz = g.box[3 * rep + 2];
        const float ibx = bx > 0.f ? 1.f / bx : 0.f, iby = by > 0.f ? 1.f / by : 0.f, ibz = bz > 0.f ? 1.f / bz : 0.f;
        const float xi = g.x[3 * i], yi = g.x[3 * i + 1], zi = g.x[3 * i + 2];
        for (int e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e) {
            const int j = __ldg(g.col + e);
            const float dx = min_img(__ldg(g.x + 3 * j) - xi, bx, ibx);
            const float dy = min_img(__ldg(g.x + 3 * j + 1) - yi, by, iby);
            const float dz = min_img(__ldg(g.x + 3 * j + 2) - zi, bz, ibz);
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < rc2)) continue;   // uniform over the warp
            const float r = sqrtf(r2), inv = 1.f / r;
            float du;
            const float fc = envelope(r * g.inv_rc, g.p, &du);
            float B[K], Y[4];
            bessel<K, false>(r, g.inv_rc, g.bnorm, B, nullptr);
            sph<1>(dx * inv, dy * inv, dz * inv, Y);
#pragma unroll
            for (int u = 0; u < CPW; ++u) {
                const float sj = __ldg(g.s0 + (size_t)j * C + lane * CPW + u);
                const float z0 = gA[0][u] * Y[0] * sj * fc;
                const float z1 = fmaf(gA[1][u], Y[1], fmaf(gA[2][u], Y[2], gA[3][u] * Y[3])) * sj * fc;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    wacc[0][k][u] = fmaf(z0, B[k], wacc[0][k][u]);
                    wacc[1][k][u] = fmaf(z1, B[k], wacc[1][k][u]);
                }
            }
        }
    }
#pragma unroll
    for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int u = 0; u < CPW; ++u) red[warp][(l * K + k) * C + lane * CPW + u] = g.nu * wacc[l][k][u];
    __syncthreads();
    for (int q = threadIdx.x; q < NW; q += blockDim.x)
        part[(size_t)blockIdx.x * NW + q] = ((red[0][q] + red[1][q]) + red[2][q]) + red[3][q];
}

__global__ void k_sum_rows(int Q, int rows, const float *__restrict__ part, float *__restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    float t = 0.f;
    for (int r = 0; r < rows; ++r) t += part[(size_t)r * Q + q];
    out[q] = t;
}

void launch_nc_layer_wgrad(int C, const NCLayerGradArgs &a, float *part, float *out, cudaStream_t st) {
    if (a.n_atoms == 0) return;
    const int blocks = std::max(1, std::min(WG_BLOCKS, (a.n_atoms + 3) / 4));
    if (C == 32) k_nc_layer_wgrad<32><<<blocks, 128, 0, st>>>(a, part);
    else if (C == 64) k_nc_layer_wgrad<64><<<blocks, 128, 0, st>>>(a, part);
    else return;
    count_launch();
    const int Q = 2 * 8 * C;
    k_sum_rows<<<(Q + 255) / 256, 256, 0, st>>>(Q, blocks, part, out);
    count_launch();
}

__global__ void k_nc_dU_part(int n, int C, int n_l, const float *__restrict__ gV, const float *__restrict__ A,
                             float *__restrict__ part, int slices) {
    const int q = threadIdx.x;   // q = t C + c
    if (q >= n_l * C) return;
    const int t = q / C, c = q - t * C;
    const int per = (n + slices - 1) / slices, a0 = blockIdx.x * per, a1 = min(n, a0 + per);
    float acc = 0.f;
    for (int i = a0; i < a1; ++i)
#pragma unroll
        for (int m = 0; m < 3; ++m) acc = fmaf(gV[((size_t)i * n_l + t) * 3 + m], A[((size_t)i * 4 + 1 + m) * C + c], acc);
    part[(size_t)blockIdx.x * n_l * C + q] = acc;
}

void launch_nc_dU(int n, int C, int n_l, const float *gV, const float *A, float *part, float *out, cudaStream_t st) {
    if (n == 0) return;
    const int slices = std::max(1, std::min(64, (n + 255) / 256));
    k_nc_dU_part<<<slices, 256, 0, st>>>(n, C, n_l, gV, A, part, slices);
    count_launch();
    k_sum_rows<<<(n_l * C + 255) / 256, 256, 0, st>>>(n_l * C, slices, part, out);
    count_launch();
}

__global__ void k_distill_residual(int n, const float *F, const float *T, float *g, float *sq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float d = F[3 * i + q] - T[3 * i + q];
        g[3 * i + q] = 2.f * d;
        s = fmaf(d, d, s);
    }
    sq[i] = s;
}

void launch_distill_residual(int n, const float *F, const float *T, float *g, float *sq, cudaStream_t st) {
    if (n == 0) return;
    k_distill_residual<<<(n + 255) / 256, 256, 0, st>>>(n, F, T, g, sq);
    count_launch();
}

// Adam (Kingma & Ba), beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected.
__global__ void k_adam(int n, float *w, const float *grad, float *m, float *v, float lr, float c1, float c2,
                       __nv_bfloat16 *w_bf, int kd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gr = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * gr, vi = 0.999f * v[i] + 0.001f * gr * gr;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    w[i] = wi;
    if (w_bf) st_split(w_bf, (size_t)(i / kd), kd, i % kd, wi);
}

void launch_adam(int n, float *w, const float *grad, float *m, float *v, float lr, int step, __nv_bfloat16 *w_bf,
                 int kd, cudaStream_t st) {
    if (n == 0) return;
    const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
    k_adam<<<(n + 255) / 256, 256, 0, st>>>(n, w, grad, m, v, lr, c1, c2, w_bf, kd);
    count_launch();
}

__global__ void k_scale_d(double *v, int n, double f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] *= f;
}

void launch_scale_d(double *v, int n, double f, cudaStream_t st) {
    if (n == 0) return;
    k_scale_d<<<(n + 255) / 256, 256, 0, st>>>(v, n, f);
    count_launch();
}

// Virial estimator of a RESPA outer step (Sec. 2, "Computation of the virial
// term in NPT"): the full force's virial at the step's end, with the fast
// force's share there replaced by its average over the inner steps.
__global__ void k_virial_estimate(double *est, const double *cons, const double *last, const double *avg, int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) est[r] = cons[r] - last[r] + avg[r];
}

void launch_virial_estimate(double *est, const double *cons, const double *last, const double *avg, int n,
                            cudaStream_t st) {
    if (n == 0) return;
    k_virial_estimate<<<(n + 255) / 256, 256, 0, st>>>(est, cons, last, avg, n);
    count_launch();
}

// Mean subtraction over each replica in three short kernels. A replica is
// cut into parts of MS_PART atoms counted from its own first atom, so every
// sum below depends only on the replica's atoms, never on which other
// replicas share the batch. Within a part, thread t adds atoms t, t + 256,
// ... in fp32 (at most four), the block then adds the thread sums in fp64 in
// a fixed tree; the per-part fp64 sums are added in part order.
constexpr int MS_PART = 1024, MS_THREADS = 256;

// part_off[r] = sum over r' < r of ceil(len_r' / MS_PART), r = 0 .. n_rep;
// net = 0 for replicas without atoms.
__global__ void k_mean_part_off(const int *__restrict__ rep_off, int n_rep, int *__restrict__ part_off,
                                double *__restrict__ net) {
    __shared__ int carry, warp_tot[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int r0 = 0; r0 < n_rep; r0 += blockDim.x) {
        const int r = r0 + threadIdx.x;
        const int len = r < n_rep ? rep_off[r + 1] - rep_off[r] : 0;
        const int v = (len + MS_PART - 1) / MS_PART;
        if (net && r < n_rep && len == 0)
            for (int c = 0; c < 3; ++c) net[3 * r + c] = 0.0;
        int inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(DMTS_FULL, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) warp_tot[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(DMTS_FULL, w, o);
                if (lane >= o) w += t;
            }
            warp_tot[lane] = w;    // inclusive over warps
        }
        __syncthreads();
        const int excl = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + inc - v;
        if (r < n_rep) part_off[r] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) part_off[n_rep] = carry;
}

// Replica r and part p of block b (b < part_off[n_rep]); false for spare blocks.
__device__ __forceinline__ bool mean_part_of(const int *part_off, int n_rep, int b, int &r, int &p) {
    if (b >= part_off[n_rep]) return false;
    int lo = 0, hi = n_rep;     // largest r with part_off[r] <= b
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (part_off[mid] <= b) lo = mid; else hi = mid;
    }
    // replicas without atoms have no parts: skip to the one that owns b
    while (part_off[lo + 1] <= b) ++lo;
    r = lo;
    p = b - part_off[lo];
    return true;
}

__global__ void __launch_bounds__(MS_THREADS) k_mean_partial(const float *__restrict__ F_in,
                                                             const int *__restrict__ rep_off,
                                                             const int *__restrict__ part_off, int n_rep,
                                                             double *__restrict__ partial, const int *__restrict__ err) {
    if (*err) return;
    int r, p;
    if (!mean_part_of(part_off, n_rep, blockIdx.x, r, p)) return;
    const int lo = rep_off[r] + p * MS_PART, hi = min(rep_off[r + 1], lo + MS_PART);
    float v[MS_PART / MS_THREADS][3];
#pragma unroll
    for (int k = 0; k < MS_PART / MS_THREADS; ++k) {
        const int i = lo + threadIdx.x + k * MS_THREADS;
        for (int c = 0; c < 3; ++c) v[k][c] = i < hi ? F_in[3 * i + c] : 0.f;
    }
    __shared__ double red[3][MS_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = 0; c < 3; ++c) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < MS_PART / MS_THREADS; ++k) t += v[k][c];
        const double d = warp_sum_d((double)t);
        if (lane == 0) red[c][wid] = d;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < MS_THREADS / 32; ++w) t += red[threadIdx.x][w];
        partial[3 * (size_t)blockIdx.x + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(MS_THREADS) k_mean_apply(const float *__restrict__ F_in, float *__restrict__ F_out,
                                                           const int *__restrict__ rep_off,
                                                           const int *__restrict__ part_off, int n_rep,
                                                           const double *__restrict__ partial,
                                                           double *__restrict__ net, const int *__restrict__ err) {
    if (*err) return;
    int r, p;
    if (!mean_part_of(part_off, n_rep, blockIdx.x, r, p)) return;
    __shared__ float mean[3];
    const int beg = rep_off[r], end = rep_off[r + 1];
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int q = part_off[r]; q < part_off[r + 1]; ++q) t += partial[3 * (size_t)q + threadIdx.x];
        if (net && p == 0) net[3 * r + threadIdx.x] = t;
        mean[threadIdx.x] = (float)(t / (double)(end - beg));
    }
    __syncthreads();
    const int lo = beg + p * MS_PART, hi = min(end, lo + MS_PART);
    const float mx = mean[0], my = mean[1], mz = mean[2];
#pragma unroll
    for (int k = 0; k < MS_PART / MS_THREADS; ++k) {
        const int i = lo + threadIdx.x + k * MS_THREADS;
        if (i < hi) {
            F_out[3 * i] = F_in[3 * i] - mx;
            F_out[3 * i + 1] = F_in[3 * i + 1] - my;
            F_out[3 * i + 2] = F_in[3 * i + 2] - mz;
        }
    }
}

size_t mean_sub_scratch_bytes(int n_atoms, int n_rep) {
    const size_t parts = (size_t)(n_atoms + MS_PART - 1) / MS_PART + (size_t)n_rep;
    return 3 * sizeof(double) * parts + sizeof(int) * ((size_t)n_rep + 1) + 64;
}

void launch_mean_part_off(const int *rep_off, int n_rep, int *part_off, cudaStream_t st) {
    if (n_rep == 0) return;
    k_mean_part_off<<<1, 1024, 0, st>>>(rep_off, n_rep, part_off, nullptr);
    count_launch();
}

void launch_mean_sub(const float *F_in, float *F_out, const int *rep_off, int n_rep, int n_atoms, double *net,
                     void *scratch, const int *err, cudaStream_t st, const int *part_off_pre) {
    if (n_rep == 0) return;
    const int parts = (n_atoms + MS_PART - 1) / MS_PART + n_rep;   // bound on the parts of all replicas
    double *partial = static_cast<double *>(scratch);
    int *part_off = reinterpret_cast<int *>(partial + 3 * (size_t)parts);
    if (part_off_pre && !net) {
        part_off = const_cast<int *>(part_off_pre);
    } else {
        k_mean_part_off<<<1, 1024, 0, st>>>(rep_off, n_rep, part_off, net);
        count_launch();
    }
    k_mean_partial<<<parts, MS_THREADS, 0, st>>>(F_in, rep_off, part_off, n_rep, partial, err);
    count_launch();
    k_mean_apply<<<parts, MS_THREADS, 0, st>>>(F_in, F_out, rep_off, part_off, n_rep, partial, net, err);
    count_launch();
}

// ------------------------------------------------ NC forces: fixed point
// One thread per atom: the head's 32.32 fixed-point force -> fp32 (F), the
// fixed-point words cleared for the next evaluation (also when the error
// word is set, so an aborted evaluation leaves nothing behind), and the
// replica's exact integer sum of the forces added to sum[r] (warp-aggregated
// 64-bit atomics; integer sums do not depend on their order).
__global__ void k_nc_convert(int n, const int *__restrict__ atom_rep, unsigned long long *__restrict__ Ffix,
                             float *__restrict__ F, unsigned long long *__restrict__ sum, unsigned *__restrict__ next) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && next) *next = 0u;   // the head's work counter, for its next launch
    const bool live = i < n;
    const int r = live ? atom_rep[i] : -1;
    long long q[3] = {0, 0, 0};
    if (live) {
        for (int c = 0; c < 3; ++c) {
            q[c] = (long long)Ffix[3 * i + c];
            Ffix[3 * i + c] = 0ull;
            F[3 * i + c] = fix_to_float(q[c]);
        }
    }
    const int leader = __ffs(__match_any_sync(DMTS_FULL, r)) - 1;
    for (int c = 0; c < 3; ++c) {
        const long long t = seg_sum_ll(q[c], r);
        if (live && (int)(threadIdx.x & 31) == leader) fix_add(sum + 3 * (size_t)r + c, t);
    }
}

void launch_nc_convert(int n, const int *atom_rep, unsigned long long *Ffix, float *F, unsigned long long *sum,
                       unsigned *next, cudaStream_t st) {
    if (n == 0) return;
    k_nc_convert<<<(n + 255) / 256, 256, 0, st>>>(n, atom_rep, Ffix, F, sum, next);
    count_launch();
}

// F_out = F - the replica's mean (from the exact sums); net (nullable) [R][3].
__global__ void k_nc_apply(int n, const int *__restrict__ atom_rep, const int *__restrict__ rep_off, int n_rep,
                           const float *__restrict__ F, float *__restrict__ F_out,
                           const unsigned long long *__restrict__ sum, double *__restrict__ net,
                           const int *__restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (net && i < 3 * n_rep) net[i] = fix_sum_to_double(sum[i]);
    if (i >= n || *err) return;
    const int r = atom_rep[i];
    const float3 m = fix_mean(sum, rep_off, r);
    F_out[3 * i] = F[3 * i] - m.x;
    F_out[3 * i + 1] = F[3 * i + 1] - m.y;
    F_out[3 * i + 2] = F[3 * i + 2] - m.z;
}

void launch_nc_apply(int n, const int *atom_rep, const int *rep_off, int n_rep, const float *F, float *F_out,
                     const unsigned long long *sum, double *net, const int *err, cudaStream_t st) {
    const int work = n > 3 * n_rep ? n : 3 * n_rep;
    if (work == 0) return;
    k_nc_apply<<<(work + 255) / 256, 256, 0, st>>>(n, atom_rep, rep_off, n_rep, F, F_out, sum, net, err);
    count_launch();
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
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f, w = 0.f;
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
            w += 0.5f * c * r2;
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
        w += 0.5f * c * r2;
    };
    for_active_canonical(g.col, g.row_ptr[a], g.row_ptr[a + 1], sh_queue[warp], lane, active, edge);
    if (g.bonds.ptr) bond_force(g.bonds, g.x, a, bx, by, bz, ibx, iby, ibz, lane, fx, fy, fz, e, &w);
    fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz); e = warp_sum(e);
    if (g.W) w = warp_sum(w);
    if (lane == 0) {
        g.F[3 * a] += fx; g.F[3 * a + 1] += fy; g.F[3 * a + 2] += fz;
        if (g.e_atom) g.e_atom[a] += e;
        if (g.W) g.W[a] += w;
    }
}

void launch_prior(const PriorArgs &a, cudaStream_t st) {
    if (a.n_atoms == 0) return;
    k_prior<<<(a.n_atoms + 3) / 4, 128, 0, st>>>(a);
    count_launch();
}

// ----------------------------------------------------------- integrator
// The closing kicks of a step, shared by the integrator and the FP64
// kinetic-energy reduction so that both form the same closed velocity:
// v += h_in a F_fast (B), then v += h_out a (F_slow - F_fast) (outer kick).
__device__ __forceinline__ void closing_b(float h, float sfx, float sfy, float sfz, float &vx, float &vy, float &vz) {
    vx = fmaf(h, sfx, vx); vy = fmaf(h, sfy, vy); vz = fmaf(h, sfz, vz);
}
__device__ __forceinline__ void outer_kick(float h, float lx, float ly, float lz, float &vx, float &vy, float &vz) {
    vx = fmaf(h, lx, vx); vy = fmaf(h, ly, vy); vz = fmaf(h, lz, vz);
}

// One thread per atom; the operations selected by `ops` run in this order:
// closing B, closing outer kick, opening outer kick, then B-A-O-A.
__global__ void k_integrate(IntegArgs g) {
    if (*g.err) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_atoms) return;
    const float am = kAccConv / g.masses[i];
    float vx = g.v[3 * i], vy = g.v[3 * i + 1], vz = g.v[3 * i + 2];
    float sfx, sfy, sfz;
    if (g.fast_pre) {
        // the fast force's pending mean subtraction, stored as the cached force
        const float3 m = fix_mean(g.fast_sum, g.rep_off, g.atom_rep[i]);
        sfx = g.fast_pre[3 * i] - m.x;
        sfy = g.fast_pre[3 * i + 1] - m.y;
        sfz = g.fast_pre[3 * i + 2] - m.z;
        g.fast_out[3 * i] = sfx; g.fast_out[3 * i + 1] = sfy; g.fast_out[3 * i + 2] = sfz;
    } else {
        sfx = g.f_fast[3 * i]; sfy = g.f_fast[3 * i + 1]; sfz = g.f_fast[3 * i + 2];
    }
    if (g.ops & OP_CLOSE_B) closing_b(g.h_in * am, sfx, sfy, sfz, vx, vy, vz);
    if (g.ops & (OP_KICK_L | OP_KICK_L2)) {
        const float h = g.h_out * am;
        const float lx = g.f_slow[3 * i] - sfx, ly = g.f_slow[3 * i + 1] - sfy, lz = g.f_slow[3 * i + 2] - sfz;
        if (g.ops & OP_KICK_L) outer_kick(h, lx, ly, lz, vx, vy, vz);
        if (g.ops & OP_KICK_L2) { vx = fmaf(h, lx, vx); vy = fmaf(h, ly, vy); vz = fmaf(h, lz, vz); }
        if (g.fl_max) {
            // disagreement monitor of the rewind procedure: max |F_L| per replica
            // (non-negative floats order like their bit patterns; NaN is larger)
            const unsigned bits = __float_as_uint(sqrtf(lx * lx + ly * ly + lz * lz));
            const int r = g.atom_rep[i];
            const unsigned same = __match_any_sync(__activemask(), r);
            const unsigned top = __reduce_max_sync(same, bits);
            if ((same & ((1u << (threadIdx.x & 31)) - 1u)) == 0u) atomicMax(g.fl_max + r, top);
        }
    }
    if (g.ops & OP_BAOA) {
        const float h = g.h_in * am;
        vx = fmaf(h, sfx, vx); vy = fmaf(h, sfy, vy); vz = fmaf(h, sfz, vz);
        float x = g.x[3 * i], y = g.x[3 * i + 1], z = g.x[3 * i + 2];
        const int r = g.atom_rep[i];
        float bs = 1.f, bp = g.h_in, bv = 1.f;   // A half-step: x <- bs x + bp v, then v <- bv v
        if (g.baro_f) {
            bs = g.baro_f[3 * r]; bp = g.baro_f[3 * r + 1]; bv = g.baro_f[3 * r + 2];
            x = fmaf(bp, vx, bs * x); y = fmaf(bp, vy, bs * y); z = fmaf(bp, vz, bs * z);
            vx *= bv; vy *= bv; vz *= bv;
            if (i == g.rep_off[r]) {
                const float s2 = bs * bs;   // both half-steps of this inner step
                g.box[3 * r] *= s2; g.box[3 * r + 1] *= s2; g.box[3 * r + 2] *= s2;
            }
        } else {
            x = fmaf(g.h_in, vx, x); y = fmaf(g.h_in, vy, y); z = fmaf(g.h_in, vz, z);
        }
        const int local = i - g.rep_off[r];
        const float3 G = gauss3(g.seed[r], g.rep_id[r], g.step[r] + g.step_add, (uint32_t)local);
        const int sp = g.species[i];
        const float c1 = g.c1[sp], c2 = g.c2[sp] / sqrtf(g.masses[i]);
        const float wx = fmaf(c1, vx, c2 * G.x), wy = fmaf(c1, vy, c2 * G.y), wz = fmaf(c1, vz, c2 * G.z);
        const float nv2 = vx * vx + vy * vy + vz * vz;
        if (g.ffl && nv2 > 0.f) {
            // Fast Forward Langevin: the speed of w, the direction of v
            const float f = sqrtf(wx * wx + wy * wy + wz * wz) / sqrtf(nv2);
            vx *= f; vy *= f; vz *= f;
        } else {
            vx = wx; vy = wy; vz = wz;
        }
        if (g.baro_f) {
            x = fmaf(bp, vx, bs * x); y = fmaf(bp, vy, bs * y); z = fmaf(bp, vz, bs * z);
            vx *= bv; vy *= bv; vz *= bv;
        } else {
            x = fmaf(g.h_in, vx, x); y = fmaf(g.h_in, vy, y); z = fmaf(g.h_in, vz, z);
        }
        if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(vx) && isfinite(vy) && isfinite(vz)))
            set_error(g.err, DMTS_E_NONFINITE);
        g.x[3 * i] = x; g.x[3 * i + 1] = y; g.x[3 * i + 2] = z;
        if (g.x_ref) {
            const float ex = x - g.x_ref[3 * i], ey = y - g.x_ref[3 * i + 1], ez = z - g.x_ref[3 * i + 2];
            if (ex * ex + ey * ey + ez * ez > g.half_skin2) *g.rebuild = 1;
        }
    }
    g.v[3 * i] = vx; g.v[3 * i + 1] = vy; g.v[3 * i + 2] = vz;
    if (g.ke) g.ke[i] = 0.5f * (vx * vx + vy * vy + vz * vz) / am;   // m v^2 / 2 in kcal/mol
}

void launch_integrate(const IntegArgs &a, cudaStream_t st) {
    if (a.n_atoms == 0) return;
    k_integrate<<<(a.n_atoms + 255) / 256, 256, 0, st>>>(a);
    count_launch();
}

// ------------------------------------------------------- thermodynamics
// K = sum_i m_i |v_i|^2 / 2 per replica with every per-atom term formed in
// FP64 from the fp32 state, summed in FP64 in a fixed order over the
// replica-local parts of MS_PART atoms (the same parts as the mean
// subtraction), so the result does not depend on the batch the replica is
// in; the velocities are first closed with the step's pending kicks
// (ThermoArgs), in the integrator's own arithmetic. One block per part, then
// one thread per replica adds its parts in order and writes
// (K, U + K, 2K / (3 n_r kB)).
__global__ void __launch_bounds__(MS_THREADS) k_thermo_part(ThermoArgs g) {
    int r, p;
    if (!mean_part_of(g.part_off, g.n_rep, blockIdx.x, r, p)) return;
    const int lo = g.rep_off[r] + p * MS_PART, hi = min(g.rep_off[r + 1], lo + MS_PART);
    double acc = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += MS_THREADS) {
        const float am = kAccConv / g.masses[i];
        float vx = g.v[3 * i], vy = g.v[3 * i + 1], vz = g.v[3 * i + 2];
        if (g.close_b || g.kick_l) {
            float sfx = g.f_fast[3 * i], sfy = g.f_fast[3 * i + 1], sfz = g.f_fast[3 * i + 2];
            if (g.fast_sum) {
                const float3 m = fix_mean(g.fast_sum, g.rep_off, r);
                sfx -= m.x; sfy -= m.y; sfz -= m.z;
            }
            if (g.close_b) closing_b(g.h_in * am, sfx, sfy, sfz, vx, vy, vz);
            if (g.kick_l)
                outer_kick(g.h_out * am, g.f_slow[3 * i] - sfx, g.f_slow[3 * i + 1] - sfy, g.f_slow[3 * i + 2] - sfz,
                           vx, vy, vz);
        }
        const double dx = vx, dy = vy, dz = vz;
        acc += 0.5 * (double)g.masses[i] * (dx * dx + dy * dy + dz * dz);
    }
    __shared__ double red[MS_THREADS / 32];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < MS_THREADS / 32; ++w) t += red[w];
        g.partial[blockIdx.x] = t;
    }
}

__global__ void k_thermo_final(ThermoArgs g) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.n_rep) return;
    double t = 0.0;
    for (int q = g.part_off[r]; q < g.part_off[r + 1]; ++q) t += g.partial[q];
    const double K = t / kAccConvD;   // amu A^2/fs^2 -> kcal/mol
    const int n = g.rep_off[r + 1] - g.rep_off[r];
    const double T = n > 0 ? 2.0 * K / (3.0 * n * kBoltzmann) : 0.0;
    const double U = g.energy[r];
    double *o = g.out + 3 * (size_t)r;
    o[0] = K; o[1] = U + K; o[2] = T;
    if (g.trace) {
        double *q = g.trace + 3 * (size_t)r;
        q[0] = K; q[1] = U + K; q[2] = T;
    }
}

size_t thermo_scratch_bytes(int n_atoms, int n_rep) {
    return sizeof(double) * ((size_t)(n_atoms + MS_PART - 1) / MS_PART + (size_t)n_rep);
}

void launch_thermo(const ThermoArgs &a, int n_atoms, int n_rep, cudaStream_t st) {
    if (n_rep == 0) return;
    const int parts = (n_atoms + MS_PART - 1) / MS_PART + n_rep;   // bound on the parts of all replicas
    k_thermo_part<<<parts, MS_THREADS, 0, st>>>(a);
    count_launch();
    k_thermo_final<<<(n_rep + 127) / 128, 128, 0, st>>>(a);
    count_launch();
}

// ---------------------------------------------------------------- barostat
// One thread per replica; open replicas (box 0) keep p_eps = 0 and plain
// drift factors. N_f = 3 n_r, W = (N_f + 3) kB T tau_P^2.
__device__ __forceinline__ double baro_force(const BaroArgs &a, int r, int n) {
    const double V = (double)a.box[3 * r] * a.box[3 * r + 1] * a.box[3 * r + 2];
    return (1.0 + 1.0 / n) * 2.0 * a.K[r] - a.wvir[r] - 3.0 * V * a.p_kcal;
}

__global__ void k_baro_start(BaroArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n_rep || *a.err) return;
    const int n = a.rep_off[r + 1] - a.rep_off[r];
    double *b = a.baro + 3 * r;
    float *f = a.baro_f + 3 * r;
    if (n == 0 || !(a.box[3 * r] > 0.f)) {
        b[0] = 0.0;
        f[0] = 1.f; f[1] = (float)a.h; f[2] = 1.f;
        return;
    }
    const double W = (3.0 * n + 3.0) * a.kT * a.tau_fs * a.tau_fs;
    if (b[2] == 0.0) {   // no estimator yet: the full force's virial
        b[1] = baro_force(a, r, n);
        b[2] = 1.0;
    }
    const double c = exp(-a.delta_outer / a.tau_fs);
    const float3 G = gauss3(a.seed[r], a.rep_id[r], a.step[r] + a.step_add, 0xFFFFFFFFu);
    double p = b[0] + 0.5 * a.delta_outer * b[1];
    p = c * p + sqrt((1.0 - c * c) * W * a.kT) * (double)G.x;
    b[0] = p;
    const double beta = p / W, alpha = (1.0 + 1.0 / n) * beta, z = beta * a.h;
    f[0] = (float)exp(z);
    f[1] = (float)(z != 0.0 ? a.h * expm1(z) / z : a.h);
    f[2] = (float)exp(-alpha * a.h);
}

__global__ void k_baro_end(BaroArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n_rep || *a.err) return;
    const int n = a.rep_off[r + 1] - a.rep_off[r];
    double *b = a.baro + 3 * r;
    if (n == 0 || !(a.box[3 * r] > 0.f)) return;
    b[1] = baro_force(a, r, n);
    b[2] = 1.0;
    b[0] += 0.5 * a.delta_outer * b[1];
}

void launch_baro_start(const BaroArgs &a, cudaStream_t st) {
    if (a.n_rep == 0) return;
    k_baro_start<<<(a.n_rep + 127) / 128, 128, 0, st>>>(a);
    count_launch();
}

void launch_baro_end(const BaroArgs &a, cudaStream_t st) {
    if (a.n_rep == 0) return;
    k_baro_end<<<(a.n_rep + 127) / 128, 128, 0, st>>>(a);
    count_launch();
}

__global__ void k_advance(uint64_t *step, int n_rep, uint64_t add, const int *err) {
    if (*err) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n_rep) step[r] += add;
}

void launch_advance_step(uint64_t *step, int n_rep, uint64_t add, const int *err, cudaStream_t st) {
    if (n_rep == 0) return;
    k_advance<<<(n_rep + 127) / 128, 128, 0, st>>>(step, n_rep, add, err);
    count_launch();
}

}  // namespace dmts
