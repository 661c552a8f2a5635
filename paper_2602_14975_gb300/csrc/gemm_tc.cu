// Node-level MLP contractions on the 5th-generation tensor cores:
// Out[M][N] = Act[M][K] x W^T with bf16 operands and an fp32 accumulator in
// tensor memory, followed by the same fused epilogues as the fp32 GEMM.
//
// One CTA (eight warps) computes a 128 x BN tile (BN a multiple of 16 that
// divides N, near 64). Warp 0 (one lane) streams K-chunks of 64 bf16 of the
// activation tile and of the weight tile into shared memory with TMA
// (128-byte swizzle), warp 1 (one lane) issues tcgen05.mma (M = 128, N = BN,
// K = 16 per instruction) into a TMEM accumulator, warp 2 owns the TMEM
// allocation; warps 0-3 read the accumulator back with tcgen05.ld (warp w
// reads rows 32w..32w+31) into shared memory and all eight warps apply the
// epilogue with coalesced accesses.
//
// Split-bf16 operands (common.cuh: rows of 2K holding hi | lo) are
// contracted in three segments of K-chunks into the same accumulator,
// hi*hi + lo*hi + hi*lo, which keeps about 16 significant bits of each
// operand while every MMA is a plain bf16 x bf16 -> fp32 instruction.
//
// Every wait on an mbarrier is bounded: on timeout the CTA records
// DMTS_E_TIMEOUT, waits (bounded) for the loads and MMAs it has issued,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "mp.cuh"
#include "ptx.cuh"
#include "tc.cuh"

namespace dmts {

namespace {

constexpr int TC_M = 128;
constexpr int TC_K = 64;             // bf16 elements per 128-byte swizzled row
constexpr int TC_STAGES = 4;
constexpr int kBNTarget = 64;      // preferred column-tile width

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ float silu_d(float v) { return v / (1.f + __expf(-v)); }
__device__ __forceinline__ float dsilu_d(float v) {
    const float sg = 1.f / (1.f + __expf(-v));
    return sg * (1.f + v * (1.f - sg));
}

// Applies the epilogue to a rows x BN tile held in shared memory. Each
// thread takes EU elements per pass (row-major, consecutive threads on
// consecutive columns) and issues all of their global loads before any
// store, so that many loads are in flight per warp.
constexpr int EU = 4;

__device__ __forceinline__ void epilogue_tile(const Epi &e, int N, int rows, int m0, int n0, int BN,
                                              const float *tile, int ld) {
    const int total = rows * BN;
    const int step = blockDim.x;
    for (int base = threadIdx.x; base < total; base += EU * step) {
        float v[EU];
        size_t o[EU];
        int n[EU], r_[EU];
        bool ok[EU];
#pragma unroll
        for (int u = 0; u < EU; ++u) {
            const int idx = base + u * step;
            ok[u] = idx < total;
            const int r = ok[u] ? idx / BN : 0, c = ok[u] ? idx - r * BN : 0;
            v[u] = ok[u] ? tile[r * ld + c] : 0.f;
            n[u] = n0 + c;
            r_[u] = r;
            o[u] = (size_t)(m0 + r) * N + n[u];
        }
        switch (e.mode) {
        case EPI_STORE:
#pragma unroll
            for (int u = 0; u < EU; ++u)
                if (ok[u]) {
                    e.out[o[u]] = v[u];
                    if (e.out_bf16) st_split(e.out_bf16, (size_t)(m0 + r_[u]), N, n[u], v[u]);
                }
            break;
        case EPI_BIAS_SILU: {
            float b[EU];
#pragma unroll
            for (int u = 0; u < EU; ++u) b[u] = ok[u] ? __ldg(e.bias + n[u]) : 0.f;
#pragma unroll
            for (int u = 0; u < EU; ++u)
                if (ok[u]) {
                    const float h = v[u] + b[u];
                    const float sv = silu_d(h);
                    if (e.H) e.H[o[u]] = h;
                    if (e.out) e.out[o[u]] = sv;
                    if (e.out_bf16) st_split(e.out_bf16, (size_t)(m0 + r_[u]), N, n[u], sv);
                }
            break;
        }
        case EPI_RESID: {
            float rs[EU], b[EU];
#pragma unroll
            for (int u = 0; u < EU; ++u) {
                rs[u] = ok[u] ? __ldg(e.res + o[u]) : 0.f;
                b[u] = ok[u] ? __ldg(e.bias + n[u]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < EU; ++u)
                if (ok[u]) {
                    const float rr = rs[u] + v[u] + b[u];
                    e.out[o[u]] = rr;
                    if (e.out_bf16) st_split(e.out_bf16, (size_t)(m0 + r_[u]), N, n[u], rr);
                }
            break;
        }
        case EPI_DSILU: {
            float h[EU];
#pragma unroll
            for (int u = 0; u < EU; ++u) h[u] = ok[u] ? __ldg(e.H + o[u]) : 0.f;
#pragma unroll
            for (int u = 0; u < EU; ++u)
                if (ok[u]) {
                    const float rr = v[u] * dsilu_d(h[u]);
                    e.out[o[u]] = rr;
                    if (e.out_bf16) st_split(e.out_bf16, (size_t)(m0 + r_[u]), N, n[u], rr);
                }
            break;
        }
        case EPI_GA: {
            const int nlm = (e.lmax + 1) * (e.lmax + 1);
            float a[EU][5];
            size_t ib[EU];
            int l0[EU], nm[EU];
#pragma unroll
            for (int u = 0; u < EU; ++u) {
                const int l = n[u] / e.C, c = n[u] - l * e.C;
                const int m = (int)(o[u] / N);
                l0[u] = l * l;
                nm[u] = ok[u] ? 2 * l + 1 : 0;
                ib[u] = ((size_t)m * nlm + l0[u]) * e.C + c;
#pragma unroll
                for (int q = 0; q < 5; ++q) a[u][q] = q < nm[u] ? __ldg(e.A + ib[u] + (size_t)q * e.C) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < EU; ++u)
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    if (q < nm[u]) e.out[ib[u] + (size_t)q * e.C] = 2.f * a[u][q] * v[u];
            break;
        }
        case EPI_READOUT: {
            float b[EU], w[EU];
#pragma unroll
            for (int u = 0; u < EU; ++u) {
                b[u] = ok[u] ? __ldg(e.bias + n[u]) : 0.f;
                w[u] = ok[u] ? __ldg(e.wo + n[u]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < EU; ++u)
                if (ok[u]) {
                    const float z = v[u] + b[u];
                    e.out[o[u]] = w[u] * silu_d(z);
                    const float gz = e.scale * w[u] * dsilu_d(z);
                    e.out2[o[u]] = gz;
                    if (e.out_bf16) st_split(e.out_bf16, (size_t)(m0 + r_[u]), N, n[u], gz);
                }
            break;
        }
        }
    }
}

// Vector form of the epilogue, used when every array it touches is 16-byte
// aligned (bf16 copies 8-byte): each thread takes groups of four
// consecutive columns of a row, so global loads and stores are 16-byte
// vectors, and the row / column of its next group follow by additions.
__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
// Four consecutive columns of a split-bf16 copy (common.cuh): the hi parts
// at p, the lo parts at p + N (N = the logical row length).
__device__ __forceinline__ void st4_split(__nv_bfloat16 *p, int N, float4 v) {
    __nv_bfloat16 h[4], l[4];
    split_bf16(v.x, h[0], l[0]);
    split_bf16(v.y, h[1], l[1]);
    split_bf16(v.z, h[2], l[2]);
    split_bf16(v.w, h[3], l[3]);
    uint2 uh, ul;
    uh.x = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
    uh.y = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
    ul.x = (uint32_t)__bfloat16_as_ushort(l[0]) | ((uint32_t)__bfloat16_as_ushort(l[1]) << 16);
    ul.y = (uint32_t)__bfloat16_as_ushort(l[2]) | ((uint32_t)__bfloat16_as_ushort(l[3]) << 16);
    *reinterpret_cast<uint2 *>(p) = uh;
    *reinterpret_cast<uint2 *>(p + N) = ul;
}
__device__ __forceinline__ float4 bias4(const float *b, int n) {
    return make_float4(__ldg(b + n), __ldg(b + n + 1), __ldg(b + n + 2), __ldg(b + n + 3));
}
__device__ __forceinline__ float4 silu4(float4 h) { return make_float4(silu_d(h.x), silu_d(h.y), silu_d(h.z), silu_d(h.w)); }

constexpr int EU4 = 2;   // groups per thread and pass

__device__ __forceinline__ void epilogue_tile_v4(const Epi &e, int N, int rows, int m0, int n0, int BN,
                                                 const float *tile, int ld) {
    const int G = BN / 4, total = rows * G, step = blockDim.x;
    const int dr = step / G, dc = step - dr * G;
    int r = threadIdx.x / G, c = threadIdx.x - (threadIdx.x / G) * G;
    const int nlm = (e.lmax + 1) * (e.lmax + 1);
    for (int base = threadIdx.x; base < total; base += EU4 * step) {
        float4 v[EU4];
        int rr[EU4], cc[EU4];
        bool ok[EU4];
#pragma unroll
        for (int u = 0; u < EU4; ++u) {
            ok[u] = base + u * step < total;
            rr[u] = r;
            cc[u] = c;
            const float *t = tile + r * ld + 4 * c;
            v[u] = ok[u] ? make_float4(t[0], t[1], t[2], t[3]) : make_float4(0.f, 0.f, 0.f, 0.f);
            r += dr;
            c += dc;
            if (c >= G) { c -= G; ++r; }
        }
        switch (e.mode) {
        case EPI_STORE:
#pragma unroll
            for (int u = 0; u < EU4; ++u)
                if (ok[u]) {
                    const size_t o = (size_t)(m0 + rr[u]) * N + n0 + 4 * cc[u];
                    st4(e.out + o, v[u]);
                    if (e.out_bf16) st4_split(e.out_bf16 + (size_t)(m0 + rr[u]) * 2 * N + n0 + 4 * cc[u], N, v[u]);
                }
            break;
        case EPI_BIAS_SILU:
#pragma unroll
            for (int u = 0; u < EU4; ++u)
                if (ok[u]) {
                    const int n = n0 + 4 * cc[u];
                    const size_t o = (size_t)(m0 + rr[u]) * N + n;
                    const float4 b = bias4(e.bias, n);
                    const float4 h = make_float4(v[u].x + b.x, v[u].y + b.y, v[u].z + b.z, v[u].w + b.w);
                    const float4 sv = silu4(h);
                    if (e.H) st4(e.H + o, h);
                    if (e.out) st4(e.out + o, sv);
                    if (e.out_bf16) st4_split(e.out_bf16 + (size_t)(m0 + rr[u]) * 2 * N + n0 + 4 * cc[u], N, sv);
                }
            break;
        case EPI_RESID: {
            float4 rs[EU4];
#pragma unroll
            for (int u = 0; u < EU4; ++u)
                rs[u] = ok[u] ? ld4(e.res + (size_t)(m0 + rr[u]) * N + n0 + 4 * cc[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < EU4; ++u)
                if (ok[u]) {
                    const int n = n0 + 4 * cc[u];
                    const size_t o = (size_t)(m0 + rr[u]) * N + n;
                    const float4 b = bias4(e.bias, n);
                    const float4 o4 = make_float4(rs[u].x + v[u].x + b.x, rs[u].y + v[u].y + b.y,
                                                  rs[u].z + v[u].z + b.z, rs[u].w + v[u].w + b.w);
                    st4(e.out + o, o4);
                    if (e.out_bf16) st4_split(e.out_bf16 + (size_t)(m0 + rr[u]) * 2 * N + n0 + 4 * cc[u], N, o4);
                }
            break;
        }
        case EPI_DSILU: {
            float4 h[EU4];
#pragma unroll
            for (int u = 0; u < EU4; ++u)
                h[u] = ok[u] ? ld4(e.H + (size_t)(m0 + rr[u]) * N + n0 + 4 * cc[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < EU4; ++u)
                if (ok[u]) {
                    const size_t o = (size_t)(m0 + rr[u]) * N + n0 + 4 * cc[u];
                    const float4 o4 = make_float4(v[u].x * dsilu_d(h[u].x), v[u].y * dsilu_d(h[u].y),
                                                  v[u].z * dsilu_d(h[u].z), v[u].w * dsilu_d(h[u].w));
                    st4(e.out + o, o4);
                    if (e.out_bf16) st4_split(e.out_bf16 + (size_t)(m0 + rr[u]) * 2 * N + n0 + 4 * cc[u], N, o4);
                }
            break;
        }
        case EPI_GA: {
            // n = l C + c: the four columns share l (C % 4 == 0)
            float4 a[EU4][5];
            size_t ib[EU4];
            int nm[EU4];
#pragma unroll
            for (int u = 0; u < EU4; ++u) {
                const int n = n0 + 4 * cc[u];
                const int l = n / e.C, cch = n - l * e.C;
                nm[u] = ok[u] ? 2 * l + 1 : 0;
                ib[u] = ((size_t)(m0 + rr[u]) * nlm + l * l) * e.C + cch;
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    a[u][q] = q < nm[u] ? ld4(e.A + ib[u] + (size_t)q * e.C) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < EU4; ++u)
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    if (q < nm[u])
                        st4(e.out + ib[u] + (size_t)q * e.C,
                            make_float4(2.f * a[u][q].x * v[u].x, 2.f * a[u][q].y * v[u].y, 2.f * a[u][q].z * v[u].z,
                                        2.f * a[u][q].w * v[u].w));
            break;
        }
        case EPI_READOUT:
#pragma unroll
            for (int u = 0; u < EU4; ++u)
                if (ok[u]) {
                    const int n = n0 + 4 * cc[u];
                    const size_t o = (size_t)(m0 + rr[u]) * N + n;
                    const float4 b = bias4(e.bias, n), w = bias4(e.wo, n);
                    const float4 z = make_float4(v[u].x + b.x, v[u].y + b.y, v[u].z + b.z, v[u].w + b.w);
                    st4(e.out + o, make_float4(w.x * silu_d(z.x), w.y * silu_d(z.y), w.z * silu_d(z.z), w.w * silu_d(z.w)));
                    const float4 gz = make_float4(e.scale * w.x * dsilu_d(z.x), e.scale * w.y * dsilu_d(z.y),
                                                  e.scale * w.z * dsilu_d(z.z), e.scale * w.w * dsilu_d(z.w));
                    st4(e.out2 + o, gz);
                    if (e.out_bf16) st4_split(e.out_bf16 + (size_t)(m0 + rr[u]) * 2 * N + n0 + 4 * cc[u], N, gz);
                }
            break;
        }
    }
}

// K-chunk k of a contraction over nseg segments (nk chunks each): segment 0
// multiplies the hi parts of both operands, segment 1 the activation's lo
// part with the weight's hi part, segment 2 the activation's hi part with
// the weight's lo part; kofs is the column where the lo parts start.
__device__ __forceinline__ void chunk_coords(int k, int nk, int kofs, int &xa, int &xb) {
    const int seg = k / nk, kc = k - seg * nk;
    xa = kc * TC_K + (seg == 1 ? kofs : 0);
    xb = kc * TC_K + (seg == 2 ? kofs : 0);
}

__global__ void __launch_bounds__(256) k_gemm_tc(const __grid_constant__ CUtensorMap tmA,
                                                 const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                                                 int BN, int tmem_cols, int n_stages, int vec, int nseg, int kofs,
                                                 Epi e, int *err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[TC_STAGES], bar_empty[TC_STAGES], bar_done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh, issued_sh, consumed_sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // column tiles in reverse order: the gA epilogue's highest-degree tiles
    // (5 loads and stores per element for l = 2) are scheduled first
    const int m0 = blockIdx.x * TC_M, n0 = (gridDim.y - 1 - blockIdx.y) * BN;
    const int nk = K / TC_K, nkt = nk * nseg;
    const uint32_t a_bytes = TC_M * TC_K * 2, b_bytes = (uint32_t)BN * TC_K * 2;
    const uint32_t stage_bytes = a_bytes + ((b_bytes + 1023u) & ~1023u);
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;   // 1024-byte aligned tiles

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_done), 1);
        abort_sh = 0;
        issued_sh = 0;
        consumed_sh = 0;
        mbar_init_fence();
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        int k = 0;
        for (; k < nkt; ++k) {
            const int s = k % n_stages;
            if (k >= n_stages && !mbar_wait(smem_u32(&bar_empty[s]), ((k / n_stages) - 1) & 1)) {
                atomicExch(&abort_sh, 1);
                break;
            }
            int xa, xb;
            chunk_coords(k, nk, kofs, xa, xb);
            const uint32_t sa = base + s * stage_bytes, sb = sa + a_bytes;
            mbar_expect_tx(smem_u32(&bar_full[s]), a_bytes + b_bytes);
            tma_load_2d(sa, &tmA, xa, m0, smem_u32(&bar_full[s]));
            tma_load_2d(sb, &tmB, xb, n0, smem_u32(&bar_full[s]));
        }
        issued_sh = k;   // loads issued; read after the block-wide barrier below
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = idesc_bf16(TC_M, BN);
        int k = 0;
        for (; k < nkt; ++k) {
            const int s = k % n_stages;
            if (!mbar_wait(smem_u32(&bar_full[s]), (k / n_stages) & 1)) {
                atomicExch(&abort_sh, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = base + s * stage_bytes, sb = sa + a_bytes;
#pragma unroll
            for (int kk = 0; kk < TC_K / 16; ++kk)
                mma_bf16(tmem, smem_desc(sa + kk * 32), smem_desc(sb + kk * 32), idesc, (k > 0 || kk > 0) ? 1u : 0u);
            mma_commit(smem_u32(&bar_empty[s]));
        }
        consumed_sh = k;   // stages whose loads landed
        // arrives once every MMA issued above has completed
        mma_commit(smem_u32(&bar_done));
    }
    __syncwarp();
    // ---- epilogue: wait for the accumulator, read it back, fused epilogue
    const bool done = mbar_wait(smem_u32(&bar_done), 0);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!__syncthreads_and(done ? 1 : 0) || abort_sh) {
        if (threadIdx.x == 0) {
            atomicCAS(err, 0, (int)DMTS_E_TIMEOUT);
            // Drain before tensor and shared memory are released: every load
            // issued but not consumed (at most one per stage, the producer
            // refills a stage only after its MMAs completed) must land, and
            // the MMAs issued must complete; each wait again bounded.
            for (int k = consumed_sh; k < issued_sh; ++k)
                mbar_wait(smem_u32(&bar_full[k % n_stages]), (k / n_stages) & 1);
            if (!done) mbar_wait(smem_u32(&bar_done), 0);
        }
    } else {
        // TMEM -> shared memory (the drained pipeline buffers): warps 0-3
        // each move their 32-lane quarter, one row per lane. Then all eight
        // warps walk the tile row-major, consecutive threads on consecutive
        // columns, so the epilogue's loads and stores are coalesced and many
        // warps hide their latency.
        const int ld = BN + 1;
        float *tile = reinterpret_cast<float *>(smem_raw + (base - smem_u32(smem_raw)));
        if (warp < 4) {
            float *wtile = tile + (size_t)warp * 32 * ld;
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
            for (int c = 0; c < BN; c += 16) {
                float v[16];
                tmem_ld16(trow + (uint32_t)c, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) wtile[lane * ld + c + q] = v[q];
            }
        }
        __syncthreads();
        const int rows = min(TC_M, M - m0);
        if (vec) epilogue_tile_v4(e, N, rows, m0, n0, BN, tile, ld);
        else epilogue_tile(e, N, rows, m0, n0, BN, tile, ld);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
}

// ------------------------------------------------------------------- host
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mutex;

bool encode_fn() {
    std::lock_guard<std::mutex> lock(g_encode_mutex);
    if (g_encode) return true;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return false;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return true;
}

// 2-D bf16 tensor map over rows x cols (row-major), box of box_rows x 64.
bool make_map(CUtensorMap *map, const void *ptr, int rows, int cols, int box_rows) {
    if (!encode_fn()) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_K, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Validity of a bf16 tensor-core contraction shape.
bool gemm_tc_supported(int N, int K) { return K % TC_K == 0 && K > 0 && N % 16 == 0 && N > 0; }

int launch_gemm_tc(int M, int N, int K, const __nv_bfloat16 *Act, const __nv_bfloat16 *Wt, const Epi &e, int *err,
                   cudaStream_t st, int split, int nseg) {
    if (M == 0) return 0;
    if (!gemm_tc_supported(N, K)) return -1;
    if (!(nseg == 1 || (split && nseg == 3))) return -1;
    const int width = split ? 2 * K : K;   // physical row length of both operands
    if (((uintptr_t)Act & 15) || ((uintptr_t)Wt & 15)) return -2;
    // column tile: the multiple of 16 dividing N closest to kBNTarget (the
    // smaller on a tie). Narrow tiles give more CTAs per SM (a smaller
    // epilogue staging tile) and more CTAs per contraction, which the
    // latency-bound epilogues of these short-K contractions need.
    int BN = 0;
    for (int b = 16; b <= 256 && b <= N; b += 16)
        if (N % b == 0 && (BN == 0 || std::abs(b - kBNTarget) < std::abs(BN - kBNTarget))) BN = b;
    if (!BN) return -1;
    // a narrow contraction (one or two column tiles) halves its tiles while
    // the grid has fewer than two CTAs per SM: these launches are bound by
    // latency, not by the second read of the activation tile (from L2)
    static int n_sm = 0;
    if (!n_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        n_sm = std::max(n_sm, 1);
    }
    const int row_tiles = (M + TC_M - 1) / TC_M;
    while (BN % 32 == 0 && (long long)row_tiles * (N / BN) < 2LL * n_sm) BN /= 2;
    int tmem_cols = 32;
    while (tmem_cols < BN) tmem_cols <<= 1;
    CUtensorMap ma, mb;
    if (!make_map(&ma, Act, M, width, TC_M) || !make_map(&mb, Wt, N, width, BN)) return -3;
    const uint32_t stage = TC_M * TC_K * 2 + ((BN * TC_K * 2 + 1023) & ~1023);
    const int n_stages = std::min(3, nseg * K / TC_K);
    const size_t tile = (size_t)TC_M * (BN + 1) * sizeof(float);   // epilogue staging
    const size_t smem = std::max((size_t)stage * n_stages, tile) + 1024;
    // per launch: the attribute belongs to the current device's context
    cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    auto al = [](const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; };
    const int vec = al(e.out, 16) && al(e.out2, 16) && al(e.H, 16) && al(e.res, 16) && al(e.A, 16) &&
                    al(e.out_bf16, 8) && (e.mode != EPI_GA || e.C % 4 == 0);
    dim3 grid((M + TC_M - 1) / TC_M, N / BN);
    k_gemm_tc<<<grid, 256, smem, st>>>(ma, mb, M, N, K, BN, tmem_cols, n_stages, vec, nseg, K, e, err);
    count_launch();
    return 0;
}

}  // namespace dmts
