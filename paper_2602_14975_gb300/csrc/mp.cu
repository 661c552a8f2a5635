// Message-passing layer: edge embedding (Bessel x envelope, real SH),
// segmented scatter-sum with one warp per receiver, and the adjoint (forces
// and feature gradients) written as an atomic-free gather over the symmetric
// neighbour list. Node-level MLP contractions: SIMT fp32 GEMM with fused
// epilogues.
#include "mp.cuh"

namespace dmts {

constexpr int MP_WARPS = 4;

// ------------------------------------------------------------------ forward
// Warp per receiver i, lane owns CPW consecutive channels c = lane*CPW + u.
// Active edges (r < rc) of the row are compacted 32 at a time into shared
// memory with their embedding (f_c B_k, Y_lm); every lane then sweeps them.
// C channels are split over SPLIT thread blocks (blockIdx.y = part): a warp
// owns CW = C / SPLIT channels, offset co = part * CW.
template <int C, int LMAX, int K, int SPLIT>
__global__ void __launch_bounds__(MP_WARPS * 32) k_mp_fwd(EdgeGeom g, LayerIO io) {
    constexpr int NL = LMAX + 1, NLM = NL * NL, CW = C / SPLIT, CPW = CW / 32;
    const int co = blockIdx.y * CW;
    __shared__ float sh_b[MP_WARPS][32][K];
    __shared__ float sh_y[MP_WARPS][32][NLM];
    __shared__ int sh_j[MP_WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wi = blockIdx.x * MP_WARPS + warp;
    if (wi >= g.n_atoms || *io.err) return;
    const int i = g.order ? __ldg(g.order + wi) : wi;   // spatially sorted: neighbours shared in cache

    float W[NL][K][CPW];
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int k = 0; k < K; ++k) ldv<CPW>(io.wrad + (l * K + k) * C + co + lane * CPW, W[l][k]);
    float acc[NLM][CPW];
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm)
#pragma unroll
        for (int u = 0; u < CPW; ++u) acc[lm][u] = 0.f;

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
            const float r = sqrtf(r2), inv = 1.f / r;
            float du;
            const float fc = envelope(r * g.inv_rc, g.p, &du);
            float B[K];
            bessel<K, false>(r, g.inv_rc, g.bnorm, B, nullptr);
#pragma unroll
            for (int k = 0; k < K; ++k) sh_b[warp][pos][k] = fc * B[k];
            float Y[NLM];
            sph<LMAX>(dx * inv, dy * inv, dz * inv, Y);
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) sh_y[warp][pos][lm] = Y[lm];
            sh_j[warp][pos] = j;
        }
        __syncwarp();
        const int na = __popc(m);
#pragma unroll 2
        for (int t = 0; t < na; ++t) {
            const int jt = sh_j[warp][t];
            float sj[CPW];
            ldv<CPW>(io.s + (size_t)jt * C + co + lane * CPW, sj);
            float b[K], y[NLM];
#pragma unroll
            for (int k = 0; k < K; ++k) b[k] = sh_b[warp][t][k];
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) y[lm] = sh_y[warp][t][lm];
#pragma unroll
            for (int u = 0; u < CPW; ++u)
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    float R = 0.f;
#pragma unroll
                    for (int k = 0; k < K; ++k) R = fmaf(W[l][k][u], b[k], R);
                    const float msg = R * sj[u];
#pragma unroll
                    for (int lm = l * l; lm < (l + 1) * (l + 1); ++lm) acc[lm][u] = fmaf(msg, y[lm], acc[lm][u]);
                }
        }
        __syncwarp();
    }
    float qv[NL][CPW];
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int u = 0; u < CPW; ++u) qv[l][u] = 0.f;
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) {
        const int l = lm == 0 ? 0 : (lm < 4 ? 1 : 2);
        float a[CPW];
#pragma unroll
        for (int u = 0; u < CPW; ++u) {
            a[u] = io.nu * acc[lm][u];
            qv[l][u] = fmaf(a[u], a[u], qv[l][u]);
        }
        stv<CPW>(io.A + ((size_t)i * NLM + lm) * C + co + lane * CPW, a);
    }
    if (LMAX >= 1 && io.V) {
        // vector part of the tensor heads, V_h = sum_c U[h][c] A[l=1][c]
        for (int h = 0; h < io.n_l; ++h) {
            float u4[CPW];
            ldv<CPW>(io.U + (size_t)h * C + co + lane * CPW, u4);
#pragma unroll
            for (int cmp = 0; cmp < 3; ++cmp) {
                float part = 0.f;
#pragma unroll
                for (int u = 0; u < CPW; ++u) part = fmaf(u4[u], io.nu * acc[1 + cmp][u], part);
                part = warp_sum(part);
                if (lane == 0) io.V[((size_t)i * io.n_l + h) * 3 + cmp] = part;
            }
        }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        stv<CPW>(io.q + (size_t)i * NL * C + l * C + co + lane * CPW, qv[l]);
        if (io.q_bf16) {
#pragma unroll
            for (int u = 0; u < CPW; ++u)
                io.q_bf16[(size_t)i * NL * C + l * C + co + lane * CPW + u] = __float2bfloat16_rn(qv[l][u]);
        }
    }
}

// ----------------------------------------------------------------- adjoint
// For atom a and each neighbour j (n = n_aj, r = r_aj), with
//   Gam[c][lm] = gA_a[lm][c] s_j[c] + (-1)^l gA_j[lm][c] s_a[c],
// the force is F_a = nu sum_j ( rho n + sum_lm beta_lm dY_lm/dd ), where
//   rho = sum_c sum_l R'_lc sum_m Gam Y_lm,  beta_lm = sum_c Gam R_lc,
// and the feature gradient of the sender role is
//   g_s_a[c] += nu sum_j sum_l (-1)^l R_lc sum_m gA_j[lm][c] Y_lm.
// (Edge j->a has d_ja = -d_aj, Y_lm(-n) = (-1)^l Y_lm(n).)
template <int C, int LMAX, int K, bool VIR>
__global__ void __launch_bounds__(MP_WARPS * 32) k_mp_bwd(EdgeGeom g, LayerIO io) {
    constexpr int NL = LMAX + 1, NLM = NL * NL, CPW = C / 32;
    constexpr int STRIDE = 2 * K + NLM + 3 * NLM + 3 + (VIR ? 1 : 0);   // b, db, Y, dY, n (, r)
    __shared__ float sh_e[MP_WARPS][32][STRIDE];
    __shared__ int sh_j[MP_WARPS][32];
    __shared__ float sh_ga[MP_WARPS][NLM][C];   // element (lm, lane*CPW+u) at [lm][u*32+lane]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wa = blockIdx.x * MP_WARPS + warp;
    if (wa >= g.n_atoms || *io.err) return;
    const int a = g.order ? __ldg(g.order + wa) : wa;

    float W[NL][K][CPW];
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int k = 0; k < K; ++k) ldv<CPW>(io.wrad + (l * K + k) * C + lane * CPW, W[l][k]);
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) {
        float t[CPW];
        ldv<CPW>(io.gA + ((size_t)a * NLM + lm) * C + lane * CPW, t);
#pragma unroll
        for (int u = 0; u < CPW; ++u) sh_ga[warp][lm][u * 32 + lane] = t[u];
    }
    float sa[CPW], gsacc[CPW];
    ldv<CPW>(io.s + (size_t)a * C + lane * CPW, sa);
#pragma unroll
    for (int u = 0; u < CPW; ++u) gsacc[u] = 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f, wv = 0.f;

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
        const unsigned m = __ballot_sync(DMTS_FULL, act);
        if (act) {
            const int pos = __popc(m & ((1u << lane) - 1u));
            float *se = sh_e[warp][pos];
            const float r = sqrtf(r2), inv = 1.f / r;
            float du;
            const float fc = envelope(r * g.inv_rc, g.p, &du);
            const float dfc = du * g.inv_rc;
            float B[K], dB[K];
            bessel<K, true>(r, g.inv_rc, g.bnorm, B, dB);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                se[k] = fc * B[k];
                se[K + k] = dfc * B[k] + fc * dB[k];
            }
            const float nx = dx * inv, ny = dy * inv, nz = dz * inv;
            float Y[NLM], dY[3 * NLM];
            sph<LMAX>(nx, ny, nz, Y);
            sph_grad<LMAX>(nx, ny, nz, inv, dY);
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) se[2 * K + lm] = Y[lm];
#pragma unroll
            for (int q = 0; q < 3 * NLM; ++q) se[2 * K + NLM + q] = dY[q];
            se[2 * K + 4 * NLM] = nx;
            se[2 * K + 4 * NLM + 1] = ny;
            se[2 * K + 4 * NLM + 2] = nz;
            if (VIR) se[2 * K + 4 * NLM + 3] = r;
            sh_j[warp][pos] = j;
        }
        __syncwarp();
        const int na = __popc(m);
        for (int t = 0; t < na; ++t) {
            const int jt = sh_j[warp][t];
            const float *se = sh_e[warp][t];
            float sj[CPW];
            ldv<CPW>(io.s + (size_t)jt * C + lane * CPW, sj);
            float gj[NLM][CPW];
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) ldv<CPW>(io.gA + ((size_t)jt * NLM + lm) * C + lane * CPW, gj[lm]);
            float y[NLM];
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) y[lm] = se[2 * K + lm];
            float rho = 0.f, beta[NLM];
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) beta[lm] = 0.f;
#pragma unroll
            for (int u = 0; u < CPW; ++u) {
                float R[NL], Rp[NL];
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        s0 = fmaf(W[l][k][u], se[k], s0);
                        s1 = fmaf(W[l][k][u], se[K + k], s1);
                    }
                    R[l] = s0;
                    Rp[l] = s1;
                }
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    const float sgn = (l & 1) ? -1.f : 1.f;
                    float tl = 0.f, wl = 0.f;
#pragma unroll
                    for (int lm = l * l; lm < (l + 1) * (l + 1); ++lm) {
                        const float gal = sh_ga[warp][lm][u * 32 + lane];
                        const float gam = fmaf(gal, sj[u], sgn * gj[lm][u] * sa[u]);
                        tl = fmaf(gam, y[lm], tl);
                        beta[lm] = fmaf(gam, R[l], beta[lm]);
                        wl = fmaf(gj[lm][u], y[lm], wl);
                    }
                    rho = fmaf(Rp[l], tl, rho);
                    gsacc[u] = fmaf(sgn * R[l], wl, gsacc[u]);
                }
            }
            const float *dY = se + 2 * K + NLM;
            float ex = rho * se[2 * K + 4 * NLM], ey = rho * se[2 * K + 4 * NLM + 1], ez = rho * se[2 * K + 4 * NLM + 2];
#pragma unroll
            for (int lm = 1; lm < NLM; ++lm) {
                ex = fmaf(beta[lm], dY[3 * lm], ex);
                ey = fmaf(beta[lm], dY[3 * lm + 1], ey);
                ez = fmaf(beta[lm], dY[3 * lm + 2], ez);
            }
            fx += ex; fy += ey; fz += ez;
            // virial proxy: each directed edge's dU/dd . d is counted from both
            // ends of the pair, hence the half
            if (VIR) wv = fmaf(0.5f * se[2 * K + 4 * NLM + 3],
                               ex * se[2 * K + 4 * NLM] + ey * se[2 * K + 4 * NLM + 1] + ez * se[2 * K + 4 * NLM + 2], wv);
        }
        __syncwarp();
    }
    fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz);
    if (VIR) wv = warp_sum(wv);
    if (lane == 0) {
        const float nu = io.nu;
        if (io.accumulate) {
            io.F[3 * a] += nu * fx; io.F[3 * a + 1] += nu * fy; io.F[3 * a + 2] += nu * fz;
            if (VIR) io.W[a] += nu * wv;
        } else {
            io.F[3 * a] = nu * fx; io.F[3 * a + 1] = nu * fy; io.F[3 * a + 2] = nu * fz;
            if (VIR) io.W[a] = nu * wv;
        }
    }
    float gin[CPW], gout[CPW];
    ldv<CPW>(io.gs_in + (size_t)a * C + lane * CPW, gin);
#pragma unroll
    for (int u = 0; u < CPW; ++u) gout[u] = fmaf(io.nu, gsacc[u], gin[u]);
    stv<CPW>(io.gs_out + (size_t)a * C + lane * CPW, gout);
    if (io.gs_out_bf16) {
#pragma unroll
        for (int u = 0; u < CPW; ++u) io.gs_out_bf16[(size_t)a * C + lane * CPW + u] = __float2bfloat16_rn(gout[u]);
    }
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

// The virial variant (io.W set) is a separate instantiation, so that the
// force-only adjoint carries no extra register or instruction.
template <int C, int LMAX>
static void bwd_c(const EdgeGeom &g, const LayerIO &io, cudaStream_t st) {
    const int blocks = (g.n_atoms + MP_WARPS - 1) / MP_WARPS;
    if (io.W)
        k_mp_bwd<C, LMAX, 8, true><<<blocks, MP_WARPS * 32, 0, st>>>(g, io);
    else
        k_mp_bwd<C, LMAX, 8, false><<<blocks, MP_WARPS * 32, 0, st>>>(g, io);
    count_launch();
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
    switch (e.mode) {
    case EPI_STORE:
        e.out[o] = v;
        if (e.out_bf16) e.out_bf16[o] = __float2bfloat16_rn(v);
        break;
    case EPI_BIAS_SILU: {
        const float h = v + e.bias[n];
        e.H[o] = h;
        const float s = silu_f(h);
        e.out[o] = s;
        if (e.out_bf16) e.out_bf16[o] = __float2bfloat16_rn(s);
        break;
    }
    case EPI_RESID: {
        const float r = e.res[o] + v + e.bias[n];
        e.out[o] = r;
        if (e.out_bf16) e.out_bf16[o] = __float2bfloat16_rn(r);
        break;
    }
    case EPI_DSILU: {
        const float r = v * dsilu_f(e.H[o]);
        e.out[o] = r;
        if (e.out_bf16) e.out_bf16[o] = __float2bfloat16_rn(r);
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
        if (e.out_bf16) e.out_bf16[o] = __float2bfloat16_rn(gz);
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
