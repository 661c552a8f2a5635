// Message-passing layer: edge embedding (Bessel x envelope, real SH),
// segmented scatter-sum with one warp per receiver, and the adjoint (forces
// and feature gradients): each pair's force once, from its lower atom, in
// fixed point; each atom's sender-role gradient gathered over its row of the
// symmetric neighbour list. Node-level MLP contractions: SIMT fp32 GEMM with
// fused epilogues.
#include <type_traits>

#include "mp.cuh"

namespace dmts {

constexpr int MP_WARPS = 4;

// ------------------------------------------------------------ channel packs
// A lane owns CPW consecutive channels. With CPW even they are processed as
// pairs in packed fp32 arithmetic (fma.rn.f32x2 / mul.rn.f32x2 of sm_100 and
// later: one instruction issues two channels, each element rounded exactly as
// fmaf / a plain product), with CPW = 1 as scalars. Quantities that multiply
// every channel alike (radial basis, harmonics) are stored in shared memory
// already duplicated into both halves of a pair.
template <int CPW>
struct Pack {
    static constexpr int W = CPW % 2 == 0 ? 2 : 1;   // channels per pack
    static constexpr int NP = CPW / W;               // packs per lane
    using T = typename std::conditional<W == 2, float2, float>::type;
};

__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float vsum(float2 v) { return v.x + v.y; }
__device__ __forceinline__ float vsum(float v) { return v; }
__device__ __forceinline__ float vget(float2 v, int h) { return h ? v.y : v.x; }
__device__ __forceinline__ float vget(float v, int) { return v; }
template <class T>
__device__ __forceinline__ T vdup(float v) {
    if constexpr (std::is_same<T, float2>::value) return make_float2(v, v);
    else return v;
}

// CPW consecutive floats at p (aligned to 4 * CPW bytes) as packs, and back.
template <int CPW, class T>
__device__ __forceinline__ void ldp(const float *p, T *v) {
    if constexpr (CPW == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = make_float2(t.x, t.y);
        v[1] = make_float2(t.z, t.w);
    } else if constexpr (CPW == 2) {
        v[0] = __ldg(reinterpret_cast<const float2 *>(p));
    } else {
        v[0] = __ldg(p);
    }
}

template <int CPW, class T>
__device__ __forceinline__ void stp(float *p, const T *v) {
    if constexpr (CPW == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    else if constexpr (CPW == 2) *reinterpret_cast<float2 *>(p) = v[0];
    else *p = v[0];
}

// ------------------------------------------------------------------ forward
// Warp per receiver i, lane owns CPW consecutive channels c = lane*CPW + u.
// Active edges (r < rc) of the row are compacted 32 at a time into shared
// memory with their embedding (f_c B_k, Y_lm); every lane then sweeps them.
// C channels are split over SPLIT thread blocks (blockIdx.y = part): a warp
// owns CW = C / SPLIT channels, offset co = part * CW.
template <int C, int LMAX, int K, int SPLIT>
__global__ void __launch_bounds__(MP_WARPS * 32) k_mp_fwd(EdgeGeom g, LayerIO io) {
    constexpr int NL = LMAX + 1, NLM = NL * NL, CW = C / SPLIT, CPW = CW / 32;
    using T = typename Pack<CPW>::T;
    constexpr int NP = Pack<CPW>::NP, PW = Pack<CPW>::W;
    constexpr int RS = (K + NLM) | 1;   // odd record stride: conflict-free writes
    constexpr int FWD_UNROLL = LMAX >= 2 ? 2 : 4;   // edges in flight per lane (registers allowing)
    const int co = blockIdx.y * CW;
    __shared__ T sh_r[MP_WARPS][32][RS];
    __shared__ int sh_j[MP_WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wi = blockIdx.x * MP_WARPS + warp;
    if (wi >= g.n_atoms || *io.err) return;
    const int i = g.order ? __ldg(g.order + wi) : wi;   // spatially sorted: neighbours shared in cache

    T W[NL][K][NP];
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int k = 0; k < K; ++k) ldp<CPW>(io.wrad + (l * K + k) * C + co + lane * CPW, W[l][k]);
    T acc[NLM][NP];
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm)
#pragma unroll
        for (int p = 0; p < NP; ++p) acc[lm][p] = vdup<T>(0.f);

    const int rep = g.atom_rep[i];
    const float bx = g.box[3 * rep], by = g.box[3 * rep + 1], bz = g.box[3 * rep + 2];
    const float ibx = bx > 0.f ? 1.f / bx : 0.f, iby = by > 0.f ? 1.f / by : 0.f, ibz = bz > 0.f ? 1.f / bz : 0.f;
    const float xi = g.x[3 * i], yi = g.x[3 * i + 1], zi = g.x[3 * i + 2];
    const float rc2 = g.rc * g.rc;
    const int beg = g.row_ptr[i], end = g.row_ptr[i + 1];
    for (int base = beg; base < end; base += 32) {
        const int e = base + lane;
        bool act = false;
        int j = 0;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
        if (e < end) {
            j = __ldg(g.col + e);
            dx = min_img(__ldg(g.x + 3 * j) - xi, bx, ibx);
            dy = min_img(__ldg(g.x + 3 * j + 1) - yi, by, iby);
            dz = min_img(__ldg(g.x + 3 * j + 2) - zi, bz, ibz);
            r2 = dx * dx + dy * dy + dz * dz;
            act = r2 < rc2;
        }
        const unsigned m = __ballot_sync(DMTS_FULL, act);
        if (act) {
            const int pos = __popc(m & ((1u << lane) - 1u));
            T *rec = sh_r[warp][pos];
            const float r = sqrtf(r2), inv = 1.f / r;
            float du;
            const float fc = envelope(r * g.inv_rc, g.p, &du);
            float B[K];
            bessel<K, false>(r, g.inv_rc, g.bnorm, B, nullptr);
#pragma unroll
            for (int k = 0; k < K; ++k) rec[k] = vdup<T>(fc * B[k]);
            float Y[NLM];
            sph<LMAX>(dx * inv, dy * inv, dz * inv, Y);
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) rec[K + lm] = vdup<T>(Y[lm]);
            sh_j[warp][pos] = j;
        }
        __syncwarp();
        const int na = __popc(m);
#pragma unroll FWD_UNROLL
        for (int t = 0; t < na; ++t) {
            const int jt = sh_j[warp][t];
            const T *rec = sh_r[warp][t];
            T sj[NP];
            ldp<CPW>(io.s + (size_t)jt * C + co + lane * CPW, sj);
            T b[K], y[NLM];
#pragma unroll
            for (int k = 0; k < K; ++k) b[k] = rec[k];
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) y[lm] = rec[K + lm];
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    T Ra = vdup<T>(0.f), Rb = vdup<T>(0.f);
#pragma unroll
                    for (int k = 0; k < K; k += 2) {
                        Ra = vfma(W[l][k][p], b[k], Ra);
                        Rb = vfma(W[l][k + 1][p], b[k + 1], Rb);
                    }
                    const T R = vadd(Ra, Rb);
                    const T msg = vmul(R, sj[p]);
#pragma unroll
                    for (int lm = l * l; lm < (l + 1) * (l + 1); ++lm) acc[lm][p] = vfma(msg, y[lm], acc[lm][p]);
                }
        }
        __syncwarp();
    }
    const T nu = vdup<T>(io.nu);
    T qv[NL][NP];
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int p = 0; p < NP; ++p) qv[l][p] = vdup<T>(0.f);
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) {
        const int l = lm == 0 ? 0 : (lm < 4 ? 1 : 2);
        T a[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            a[p] = vmul(nu, acc[lm][p]);
            qv[l][p] = vfma(a[p], a[p], qv[l][p]);
        }
        if (io.A) stp<CPW>(io.A + ((size_t)i * NLM + lm) * C + co + lane * CPW, a);
    }
    if (LMAX >= 1 && io.V) {
        // vector part of the tensor heads, V_h = sum_c U[h][c] A[l=1][c]
        for (int h = 0; h < io.n_l; ++h) {
            T u4[NP];
            ldp<CPW>(io.U + (size_t)h * C + co + lane * CPW, u4);
#pragma unroll
            for (int cmp = 0; cmp < 3; ++cmp) {
                float part = 0.f;
#pragma unroll
                for (int p = 0; p < NP; ++p)
#pragma unroll
                    for (int hh = 0; hh < PW; ++hh)
                        part = fmaf(vget(u4[p], hh), io.nu * vget(acc[1 + cmp][p], hh), part);
                part = warp_sum(part);
                if (lane == 0) io.V[(size_t)i * nc_v_stride(io.n_l) + h * 3 + cmp] = part;
            }
        }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        stp<CPW>(io.q + (size_t)i * NL * C + l * C + co + lane * CPW, qv[l]);
        if (io.q_bf16) {
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int hh = 0; hh < PW; ++hh)
                    st_split(io.q_bf16, i, NL * C, l * C + co + lane * CPW + p * PW + hh, vget(qv[l][p], hh));
        }
    }
}

// ----------------------------------------------------------------- adjoint
// For atom a and a neighbour j (n = n_aj, r = r_aj), with
//   Gam[c][lm] = gA_a[lm][c] s_j[c] + (-1)^l gA_j[lm][c] s_a[c],
// the pair's force on a (both edges a <- j and j <- a) is
//   f_aj = nu ( rho n + sum_lm beta_lm dY_lm/dd ),
//   rho = sum_c sum_l R'_lc sum_m Gam Y_lm,  beta_lm = sum_c Gam R_lc,
// and the feature gradient of the sender role is
//   g_s_a[c] += nu sum_j sum_l (-1)^l R_lc sum_m gA_j[lm][c] Y_lm.
// Edge j -> a has d_ja = -d_aj and Y_lm(-n) = (-1)^l Y_lm(n), so
// Gam_ja = (-1)^l Gam_aj and dY_lm/dd at -d is -(-1)^l dY_lm/dd at d: the
// pair terms are antisymmetric, f_ja = -f_aj. Each pair's force is formed
// once, by the warp of its lower atom a < j, and enters F_a with + and F_j
// with -, in 32.32 fixed point (exact, order-independent sums; every pair's
// two terms cancel exactly), and so does its virial term. A lower
// neighbour j < a contributes only its sender-role term to g_s_a (R, no R',
// no force), and nothing in a layer without that gradient.
//
// Shared memory per block (one warp; 21.4 KB at C = 128, l_max = 2): 32 edge
// records of packs (f_c B_k, its r-derivative, Y_lm) and of scalars
// (dY_lm/dd, n, and r for the virial), the receiver's gA_a as packs, the 32
// neighbour indices, and the lanes' shares of the force of FT pairs
// (transposed so that one lane adds up each pair).
constexpr int FT = 16;   // pairs per force reduction
// One warp per block: how many upper neighbours an atom has varies from atom
// to atom, and a block keeps its registers and shared memory until its
// slowest warp is done, so single-warp blocks keep the SM's eight warp slots
// busy (255 registers a thread allow eight warps per SM either way).
constexpr int BWD_WARPS = 1;

template <int C, int LMAX, int K, bool VIR>
struct BwdSmem {
    static constexpr int NL = LMAX + 1, NLM = NL * NL, CPW = C / 32;
    using T = typename Pack<CPW>::T;
    static constexpr int NP = Pack<CPW>::NP;
    static constexpr int RS = (2 * K + NLM) | 1;
    static constexpr int GS = (3 * NLM + 3 + (VIR ? 1 : 0)) | 1;
    static constexpr size_t r_bytes = sizeof(T) * BWD_WARPS * 32 * RS;
    static constexpr size_t ga_bytes = sizeof(T) * BWD_WARPS * NLM * NP * 32;
    static constexpr size_t g_bytes = sizeof(float) * BWD_WARPS * 32 * GS;
    static constexpr size_t j_bytes = sizeof(int) * BWD_WARPS * 32;
    static constexpr size_t f_bytes = sizeof(float) * BWD_WARPS * 3 * FT * 33;
    static constexpr size_t bytes = r_bytes + ga_bytes + g_bytes + j_bytes + f_bytes;
};

// SG = false (io.gs_out == nullptr) skips the sender-role gradient: the
// first layer's input features are the species embedding, constant in the
// positions, so nothing consumes it there.
template <int C, int LMAX, int K, bool VIR, bool SG>
__global__ void __launch_bounds__(BWD_WARPS * 32) k_mp_bwd(EdgeGeom g, LayerIO io) {
    using S = BwdSmem<C, LMAX, K, VIR>;
    using T = typename S::T;
    constexpr int NL = S::NL, NLM = S::NLM, CPW = S::CPW, NP = S::NP, PW = Pack<CPW>::W;
    constexpr int RS = S::RS, GS = S::GS;
    extern __shared__ __align__(16) unsigned char mp_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T (*sh_r)[RS] = reinterpret_cast<T (*)[RS]>(mp_smem) + warp * 32;
    T (*sh_ga)[NP * 32] = reinterpret_cast<T (*)[NP * 32]>(mp_smem + S::r_bytes) + warp * NLM;
    float (*sh_g)[GS] = reinterpret_cast<float (*)[GS]>(mp_smem + S::r_bytes + S::ga_bytes) + warp * 32;
    int *sh_j = reinterpret_cast<int *>(mp_smem + S::r_bytes + S::ga_bytes + S::g_bytes) + warp * 32;
    float (*sh_f)[FT][33] =
        reinterpret_cast<float (*)[FT][33]>(mp_smem + S::r_bytes + S::ga_bytes + S::g_bytes + S::j_bytes) + warp * 3;
    const int wa = blockIdx.x * BWD_WARPS + warp;
    if (wa >= g.n_atoms || *io.err) return;
    const int a = g.order ? __ldg(g.order + wa) : wa;

    T W[NL][K][NP];
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int k = 0; k < K; ++k) ldp<CPW>(io.wrad + (l * K + k) * C + lane * CPW, W[l][k]);
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) {
        T t[NP];
        ldp<CPW>(io.gA + ((size_t)a * NLM + lm) * C + lane * CPW, t);
#pragma unroll
        for (int p = 0; p < NP; ++p) sh_ga[lm][p * 32 + lane] = t[p];
    }
    T sa[NP], san[NP], gse[NP], gso[NP];   // s_a, -s_a; sender-role sums over even and odd l
    ldp<CPW>(io.s + (size_t)a * C + lane * CPW, sa);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        san[p] = vneg(sa[p]);
        gse[p] = vdup<T>(0.f);
        gso[p] = vdup<T>(0.f);
    }
    // a's side of its pairs, fixed point (on the lanes that add up a pair)
    long long oa[3] = {0, 0, 0}, ow = 0;
    bool bad = false;   // a pair term outside the fixed-point range (or not finite)

    const int rep = g.atom_rep[a];
    const float bx = g.box[3 * rep], by = g.box[3 * rep + 1], bz = g.box[3 * rep + 2];
    const float ibx = bx > 0.f ? 1.f / bx : 0.f, iby = by > 0.f ? 1.f / by : 0.f, ibz = bz > 0.f ? 1.f / bz : 0.f;
    const float xa = g.x[3 * a], ya = g.x[3 * a + 1], za = g.x[3 * a + 2];
    const float rc2 = g.rc * g.rc;
    const int beg = g.row_ptr[a], end = g.row_ptr[a + 1];
    __syncwarp();
    for (int base = beg; base < end; base += 32) {
        const int e = base + lane;
        bool act = false;
        int j = 0;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
        if (e < end) {
            j = __ldg(g.col + e);
            dx = min_img(__ldg(g.x + 3 * j) - xa, bx, ibx);
            dy = min_img(__ldg(g.x + 3 * j + 1) - ya, by, iby);
            dz = min_img(__ldg(g.x + 3 * j + 2) - za, bz, ibz);
            r2 = dx * dx + dy * dy + dz * dz;
            act = r2 < rc2;
        }
        // lower neighbours (j < a) first, then the upper ones (the pairs this
        // warp owns): rows are ascending, so g_s_a takes its terms in row
        // order whatever the chunk boundaries (which move with the list's
        // skin entries)
        const bool up = act && j > a, lo = SG && act && j < a;
        const unsigned mu = __ballot_sync(DMTS_FULL, up), ml = __ballot_sync(DMTS_FULL, lo);
        const int n_up = __popc(mu), n_lo = __popc(ml);
        if (up || lo) {
            const unsigned lt = (1u << lane) - 1u;
            const int pos = lo ? __popc(ml & lt) : n_lo + __popc(mu & lt);
            T *rec = sh_r[pos];
            float *ge = sh_g[pos];
            const float r = sqrtf(r2), inv = 1.f / r;
            float du;
            const float fc = envelope(r * g.inv_rc, g.p, &du);
            const float dfc = du * g.inv_rc;
            float B[K], dB[K];
            bessel<K, true>(r, g.inv_rc, g.bnorm, B, dB);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                rec[k] = vdup<T>(fc * B[k]);
                rec[K + k] = vdup<T>(dfc * B[k] + fc * dB[k]);
            }
            const float nx = dx * inv, ny = dy * inv, nz = dz * inv;
            float Y[NLM], dY[3 * NLM];
            sph<LMAX>(nx, ny, nz, Y);
            sph_grad<LMAX>(nx, ny, nz, inv, dY);
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) rec[2 * K + lm] = vdup<T>(Y[lm]);
#pragma unroll
            for (int q = 0; q < 3 * NLM; ++q) ge[q] = dY[q];
            ge[3 * NLM] = nx;
            ge[3 * NLM + 1] = ny;
            ge[3 * NLM + 2] = nz;
            if (VIR) ge[3 * NLM + 3] = r;
            sh_j[pos] = j;
        }
        __syncwarp();
        if (SG) {
            // lower neighbours: the sender-role gradient only
#pragma unroll 2
            for (int t = 0; t < n_lo; ++t) {
                const int jt = sh_j[t];
                const T *rec = sh_r[t];
                T gj[NLM][NP];
#pragma unroll
                for (int lm = 0; lm < NLM; ++lm) ldp<CPW>(io.gA + ((size_t)jt * NLM + lm) * C + lane * CPW, gj[lm]);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
#pragma unroll
                    for (int l = 0; l < NL; ++l) {
                        T s0 = vdup<T>(0.f), s2 = vdup<T>(0.f);
#pragma unroll
                        for (int k = 0; k < K; k += 2) {
                            s0 = vfma(W[l][k][p], rec[k], s0);
                            s2 = vfma(W[l][k + 1][p], rec[k + 1], s2);
                        }
                        const T R = vadd(s0, s2);
                        T wl = vdup<T>(0.f);
#pragma unroll
                        for (int lm = l * l; lm < (l + 1) * (l + 1); ++lm) wl = vfma(gj[lm][p], rec[2 * K + lm], wl);
                        if (l & 1) gso[p] = vfma(R, wl, gso[p]);
                        else gse[p] = vfma(R, wl, gse[p]);
                    }
                }
            }
        }
        for (int t0 = n_lo; t0 < n_lo + n_up; t0 += FT) {
            const int t1 = min(n_lo + n_up, t0 + FT);
#pragma unroll 2
            for (int t = t0; t < t1; ++t) {
                const int jt = sh_j[t];
                const T *rec = sh_r[t];
                const float *ge = sh_g[t];
                T sj[NP];
                ldp<CPW>(io.s + (size_t)jt * C + lane * CPW, sj);
                T gj[NLM][NP];
#pragma unroll
                for (int lm = 0; lm < NLM; ++lm) ldp<CPW>(io.gA + ((size_t)jt * NLM + lm) * C + lane * CPW, gj[lm]);
                T y[NLM];
#pragma unroll
                for (int lm = 0; lm < NLM; ++lm) y[lm] = rec[2 * K + lm];
                T rho = vdup<T>(0.f), beta[NLM];
#pragma unroll
                for (int lm = 0; lm < NLM; ++lm) beta[lm] = vdup<T>(0.f);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    T R[NL], Rp[NL];
#pragma unroll
                    for (int l = 0; l < NL; ++l) {
                        T s0 = vdup<T>(0.f), s1 = vdup<T>(0.f), s2 = vdup<T>(0.f), s3 = vdup<T>(0.f);
#pragma unroll
                        for (int k = 0; k < K; k += 2) {
                            s0 = vfma(W[l][k][p], rec[k], s0);
                            s1 = vfma(W[l][k][p], rec[K + k], s1);
                            s2 = vfma(W[l][k + 1][p], rec[k + 1], s2);
                            s3 = vfma(W[l][k + 1][p], rec[K + k + 1], s3);
                        }
                        R[l] = vadd(s0, s2);
                        Rp[l] = vadd(s1, s3);
                    }
#pragma unroll
                    for (int l = 0; l < NL; ++l) {
                        const T sas = (l & 1) ? san[p] : sa[p];
                        T tl = vdup<T>(0.f), wl = vdup<T>(0.f);
#pragma unroll
                        for (int lm = l * l; lm < (l + 1) * (l + 1); ++lm) {
                            const T gam = vfma(sh_ga[lm][p * 32 + lane], sj[p], vmul(gj[lm][p], sas));
                            tl = vfma(gam, y[lm], tl);
                            beta[lm] = vfma(gam, R[l], beta[lm]);
                            if (SG) wl = vfma(gj[lm][p], y[lm], wl);
                        }
                        rho = vfma(Rp[l], tl, rho);
                        if (SG) {
                            if (l & 1) gso[p] = vfma(R[l], wl, gso[p]);
                            else gse[p] = vfma(R[l], wl, gse[p]);
                        }
                    }
                }
                // this lane's share (its channels) of the pair's force on a
                const float rh = vsum(rho);
                float ex = rh * ge[3 * NLM], ey = rh * ge[3 * NLM + 1], ez = rh * ge[3 * NLM + 2];
#pragma unroll
                for (int lm = 1; lm < NLM; ++lm) {
                    const float bl = vsum(beta[lm]);
                    ex = fmaf(bl, ge[3 * lm], ex);
                    ey = fmaf(bl, ge[3 * lm + 1], ey);
                    ez = fmaf(bl, ge[3 * lm + 2], ez);
                }
                sh_f[0][t - t0][lane] = ex;
                sh_f[1][t - t0][lane] = ey;
                sh_f[2][t - t0][lane] = ez;
            }
            __syncwarp();
            // pair t0 + u: lanes u and u + 16 add up lanes 0-15 and 16-31 of
            // its shares (conflict-free: row stride 33), then lane u the two
            // halves, in a fixed order
            const int u = lane & (FT - 1), h = lane / FT;
            const bool own = t0 + u < t1;
            float px = 0.f, py = 0.f, pz = 0.f;
            if (own) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    px += sh_f[0][u][16 * h + q];
                    py += sh_f[1][u][16 * h + q];
                    pz += sh_f[2][u][16 * h + q];
                }
            }
            px += __shfl_down_sync(DMTS_FULL, px, 16);
            py += __shfl_down_sync(DMTS_FULL, py, 16);
            pz += __shfl_down_sync(DMTS_FULL, pz, 16);
            if (own && h == 0) {
                const int jt = sh_j[t0 + u];
                px *= io.nu;
                py *= io.nu;
                pz *= io.nu;
                if (fix_ok(px) && fix_ok(py) && fix_ok(pz)) {
                    const long long qx = to_fix(px), qy = to_fix(py), qz = to_fix(pz);
                    oa[0] += qx;
                    oa[1] += qy;
                    oa[2] += qz;
                    unsigned long long *fj = io.Ffix + 3 * (size_t)jt;
                    fix_add(fj, -qx);
                    fix_add(fj + 1, -qy);
                    fix_add(fj + 2, -qz);
                    if (VIR) {
                        // virial proxy: dU/dd . d of the pair, half to each end
                        const float *ge = sh_g[t0 + u];
                        const float wp = 0.5f * ge[3 * NLM + 3] * (px * ge[3 * NLM] + py * ge[3 * NLM + 1] + pz * ge[3 * NLM + 2]);
                        if (fix_ok(wp)) {
                            const long long qw = to_fix(wp);
                            ow += qw;
                            fix_add(io.Wfix + jt, qw);
                        } else {
                            bad = true;
                        }
                    }
                } else {
                    bad = true;
                }
            }
            __syncwarp();
        }
        __syncwarp();
    }
    // a's side: the integer sums of the lanes that added up its pairs
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        oa[0] += __shfl_xor_sync(DMTS_FULL, oa[0], o);
        oa[1] += __shfl_xor_sync(DMTS_FULL, oa[1], o);
        oa[2] += __shfl_xor_sync(DMTS_FULL, oa[2], o);
        if (VIR) ow += __shfl_xor_sync(DMTS_FULL, ow, o);
    }
    if (__any_sync(DMTS_FULL, bad) && lane == 0) set_error(io.err, (int)DMTS_E_NONFINITE);
    if (lane == 0) {
        unsigned long long *fa = io.Ffix + 3 * (size_t)a;
        fix_add(fa, oa[0]);
        fix_add(fa + 1, oa[1]);
        fix_add(fa + 2, oa[2]);
        if (VIR) fix_add(io.Wfix + a, ow);
    }
    if (!SG) return;
    T gin[NP], gout[NP];
    ldp<CPW>(io.gs_in + (size_t)a * C + lane * CPW, gin);
#pragma unroll
    for (int p = 0; p < NP; ++p) gout[p] = vfma(vdup<T>(io.nu), vsub(gse[p], gso[p]), gin[p]);
    stp<CPW>(io.gs_out + (size_t)a * C + lane * CPW, gout);
    if (io.gs_out_bf16) {
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int hh = 0; hh < PW; ++hh)
                st_split(io.gs_out_bf16, a, C, lane * CPW + p * PW + hh, vget(gout[p], hh));
    }
}

// One thread per atom: the adjoint's fixed-point forces (and virial) -> fp32,
// the words cleared for the next evaluation (also after an aborted one).
__global__ void k_fix_convert(int n, unsigned long long *__restrict__ Ffix, float *__restrict__ F,
                              unsigned long long *__restrict__ Wfix, float *__restrict__ W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long q = (long long)Ffix[3 * (size_t)i + c];
        Ffix[3 * (size_t)i + c] = 0ull;
        F[3 * (size_t)i + c] = fix_to_float(q);
    }
    if (Wfix) {
        const long long q = (long long)Wfix[i];
        Wfix[i] = 0ull;
        W[i] = fix_to_float(q);
    }
}

void launch_fix_convert(int n, unsigned long long *Ffix, float *F, unsigned long long *Wfix, float *W,
                        cudaStream_t st) {
    if (n == 0) return;
    k_fix_convert<<<(n + 255) / 256, 256, 0, st>>>(n, Ffix, F, Wfix, W);
    count_launch();
}

// In the forward pass 128 channels are split over two blocks (64 per warp):
// half the registers, twice the warps in flight to hide the neighbour loads.
// The tensor-head vectors V sum over all channels, so a launch that writes V
// keeps the channels in one warp.
template <int C, int LMAX>
static void fwd_c(const EdgeGeom &g, const LayerIO &io, cudaStream_t st) {
    constexpr int SP = C >= 128 ? 2 : 1;
    const int blocks = (g.n_atoms + MP_WARPS - 1) / MP_WARPS;
    if (SP > 1 && !io.V)
        k_mp_fwd<C, LMAX, 8, SP><<<dim3(blocks, SP), MP_WARPS * 32, 0, st>>>(g, io);
    else
        k_mp_fwd<C, LMAX, 8, 1><<<blocks, MP_WARPS * 32, 0, st>>>(g, io);
    count_launch();
}

template <int C, int LMAX, bool VIR, bool SG>
static void bwd_launch(const EdgeGeom &g, const LayerIO &io, cudaStream_t st) {
    constexpr size_t smem = BwdSmem<C, LMAX, 8, VIR>::bytes;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_mp_bwd<C, LMAX, 8, VIR, SG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int blocks = (g.n_atoms + BWD_WARPS - 1) / BWD_WARPS;
    k_mp_bwd<C, LMAX, 8, VIR, SG><<<blocks, BWD_WARPS * 32, smem, st>>>(g, io);
    count_launch();
}

// The virial variant (io.Wfix set) and the variant without the sender-role
// gradient (io.gs_out null) are separate instantiations, so that each
// carries no register or instruction it does not use.
template <int C, int LMAX>
static void bwd_c(const EdgeGeom &g, const LayerIO &io, cudaStream_t st) {
    const bool gs = io.gs_out != nullptr;
    if (io.Wfix) gs ? bwd_launch<C, LMAX, true, true>(g, io, st) : bwd_launch<C, LMAX, true, false>(g, io, st);
    else gs ? bwd_launch<C, LMAX, false, true>(g, io, st) : bwd_launch<C, LMAX, false, false>(g, io, st);
}

#define DMTS_DISPATCH(FN, C, LMAX, ...)                          \
    do {                                                         \
        if ((C) == 32 && (LMAX) == 0) FN<32, 0>(__VA_ARGS__);    \
        else if ((C) == 32 && (LMAX) == 1) FN<32, 1>(__VA_ARGS__); \
        else if ((C) == 32 && (LMAX) == 2) FN<32, 2>(__VA_ARGS__); \
        else if ((C) == 64 && (LMAX) == 0) FN<64, 0>(__VA_ARGS__); \
        else if ((C) == 64 && (LMAX) == 1) FN<64, 1>(__VA_ARGS__); \
        else if ((C) == 64 && (LMAX) == 2) FN<64, 2>(__VA_ARGS__); \
        else if ((C) == 128 && (LMAX) == 0) FN<128, 0>(__VA_ARGS__); \
        else if ((C) == 128 && (LMAX) == 1) FN<128, 1>(__VA_ARGS__); \
        else if ((C) == 128 && (LMAX) == 2) FN<128, 2>(__VA_ARGS__); \
    } while (0)

void launch_mp_fwd(int C, int lmax, int K, const EdgeGeom &g, const LayerIO &io, cudaStream_t st) {
    (void)K;
    if (g.n_atoms == 0) return;
    DMTS_DISPATCH(fwd_c, C, lmax, g, io, st);
}

void launch_mp_bwd(int C, int lmax, int K, const EdgeGeom &g, const LayerIO &io, cudaStream_t st) {
    (void)K;
    if (g.n_atoms == 0) return;
    DMTS_DISPATCH(bwd_c, C, lmax, g, io, st);
}

// -------------------------------------------------------------------- GEMM
constexpr int GM = 64, GN = 64, GK = 16;

__device__ __forceinline__ void epilogue(const Epi &e, int N, int m, int n, float v) {
    const size_t o = (size_t)m * N + n;
    // bf16 copies are split hi/lo rows of width 2N (common.cuh)
    switch (e.mode) {
    case EPI_STORE:
        e.out[o] = v;
        if (e.out_bf16) st_split(e.out_bf16, m, N, n, v);
        break;
    case EPI_BIAS_SILU: {
        const float h = v + e.bias[n];
        if (e.H) e.H[o] = h;
        const float s = silu_f(h);
        if (e.out) e.out[o] = s;
        if (e.out_bf16) st_split(e.out_bf16, m, N, n, s);
        break;
    }
    case EPI_RESID: {
        const float r = e.res[o] + v + e.bias[n];
        e.out[o] = r;
        if (e.out_bf16) st_split(e.out_bf16, m, N, n, r);
        break;
    }
    case EPI_DSILU: {
        const float r = v * dsilu_f(e.H[o]);
        e.out[o] = r;
        if (e.out_bf16) st_split(e.out_bf16, m, N, n, r);
        break;
    }
    case EPI_GA: {
        const int l = n / e.C, c = n - l * e.C;
        const int nlm = (e.lmax + 1) * (e.lmax + 1);
        for (int lm = l * l; lm < (l + 1) * (l + 1); ++lm) {
            const size_t idx = ((size_t)m * nlm + lm) * e.C + c;
            e.out[idx] = 2.f * e.A[idx] * v;
        }
        break;
    }
    case EPI_READOUT: {
        const float z = v + e.bias[n];
        e.out[o] = e.wo[n] * silu_f(z);
        const float gz = e.scale * e.wo[n] * dsilu_f(z);
        e.out2[o] = gz;
        if (e.out_bf16) st_split(e.out_bf16, m, N, n, gz);
        break;
    }
    }
}

// 64x64 tile, 256 threads, 4x4 outputs per thread.
__global__ void __launch_bounds__(256) k_gemm_f32(int M, int N, int K, const float *__restrict__ Act,
                                                  const float *__restrict__ W, int trans, Epi e) {
    __shared__ float As[GK][GM + 4];
    __shared__ float Bs[GK][GN + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        // A tile: GM x GK = 1024 values, 4 per thread
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int idx = tid + t * 256;
            const int mm = idx / GK, kk = idx % GK;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? Act[(size_t)gm * K + gk] : 0.f;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int idx = tid + t * 256;
            if (trans) {
                const int nn = idx / GK, kk = idx % GK;
                const int gn = n0 + nn, gk = k0 + kk;
                Bs[kk][nn] = (gn < N && gk < K) ? W[(size_t)gn * K + gk] : 0.f;
            } else {
                const int kk = idx / GN, nn = idx % GN;
                const int gn = n0 + nn, gk = k0 + kk;
                Bs[kk][nn] = (gn < N && gk < K) ? W[(size_t)gk * N + gn] : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty * 4 + q];
                b[q] = Bs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int m = m0 + ty * 4 + p, n = n0 + tx * 4 + q;
            if (m < M && n < N) epilogue(e, N, m, n, acc[p][q]);
        }
}

void launch_gemm_f32(int M, int N, int K, const float *Act, const float *W, int trans, const Epi &e,
                     cudaStream_t st) {
    if (M == 0) return;
    dim3 grid((N + GN - 1) / GN, (M + GM - 1) / GM);
    k_gemm_f32<<<grid, 256, 0, st>>>(M, N, K, Act, W, trans, e);
    count_launch();
}

// -------------------------------------------------- per-replica FP64 sums
__global__ void k_replica_sum(const float *__restrict__ v, const int *__restrict__ rep_off,
                              double *__restrict__ out, int accumulate) {
    __shared__ double red[32];
    const int r = blockIdx.x;
    const int beg = rep_off[r], end = rep_off[r + 1];
    double acc = 0.0;
    const int stride = blockDim.x;
    for (int i0 = beg + threadIdx.x; i0 < end; i0 += 8 * stride) {
        float t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = i0 + u * stride < end ? v[i0 + u * stride] : 0.f;
        float b = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) b += t[u];
        acc += (double)b;
    }
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        t = warp_sum_d(t);
        if (threadIdx.x == 0) out[r] = accumulate ? out[r] + t : t;
    }
}

void launch_replica_sum(const float *v, const int *rep_off, int n_rep, double *out, int accumulate,
                        cudaStream_t st) {
    if (n_rep == 0) return;
    k_replica_sum<<<n_rep, 1024, 0, st>>>(v, rep_off, out, accumulate);
    count_launch();
}

}  // namespace dmts
