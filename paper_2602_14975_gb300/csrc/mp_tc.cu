// Forward message-passing layer with the radial contraction on the tensor
// cores (models with split-bf16 contractions, C = 128 channels, K = 8).
//
// For receiver i and each active edge e = (i, j) the layer needs
//   R_lc(e) = sum_k W_lkc f_c(r) B_k(r)                       (radial)
//   A_i[lm][c] = nu sum_e R_lc(e) s_j[c] Y_lm(e)              (messages)
// The radial contraction is a product of the layer's [C x K] weights with
// the edges' [K] basis vectors: one tcgen05.mma per l with the C = 128
// channels as the M = 128 rows (TMEM lanes) and 32 edges as N columns. The
// rest runs on the CUDA cores with one thread per channel (thread t reads
// TMEM lane t), two edges at a time in packed fp32.
//
// Operands are split-bf16 (common.cuh) and concatenated along K, so one
// K = 32 product holds hi*hi + lo*hi + hi*lo:
//   A row c (weights): W_hi[0..7] | W_lo[0..7] | W_hi[0..7] | 0
//   B row e (edge):    b_hi[0..7] | b_hi[0..7] | b_lo[0..7] | 0
// (nseg = 1 keeps W_hi alone: hi*hi only). Rows are 128-byte-swizzled
// K-major tiles: l = 0 and 1 share a weight tile (bytes 0-63 and 64-127 of
// each row, two K = 16 steps each), and every basis row holds the edge's
// 64 bytes twice, so that each l's MMA starts at its own half.
//
// One CTA of 128 threads (four per SM) owns a TMEM accumulator of 128
// columns and processes receivers in cell order (grid-stride). Per
// receiver, 96 candidates of its row at a time are tested; the active ones
// are compacted into shared memory (basis row for the MMA, Y_lm, neighbour
// index), then each chunk of 32 is contracted and consumed. Every mbarrier wait is
// bounded: on timeout the CTA records DMTS_E_TIMEOUT, waits (bounded) for
// the MMAs it issued, frees its tensor memory and returns.
#include <algorithm>

#include "mp.cuh"
#include "ptx.cuh"
#include "tc.cuh"

namespace dmts {

namespace {

constexpr int TF_C = 128;        // channels = TMEM lanes = threads per CTA
constexpr int TF_K = 8;          // radial basis functions
constexpr int TF_PASS = 96;      // candidates tested per pass (one per thread of the first three warps)
constexpr int TF_CHUNK = 32;     // edges per MMA (N)
constexpr int TF_TMEM = 128;     // TMEM columns: (l_max + 1) x 32 <= 96

template <int LMAX>
struct FwdTcSmem {
    static constexpr int NL = LMAX + 1;
    // weights: l = 2j and 2j + 1 share tile j (K-chunks 0-3 and 4-7 of its 128-byte rows)
    static constexpr uint32_t a_bytes = ((NL + 1) / 2) * TF_C * 128;
    static constexpr uint32_t b_bytes = TF_PASS * 128;        // basis rows of one pass
    static constexpr size_t bytes = a_bytes + b_bytes + 1024;  // + alignment slack
};

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Writes the 16-byte chunk j of row r of a swizzled tile.
__device__ __forceinline__ void st_chunk(uint8_t *tile, int r, int j, uint4 v) {
    *reinterpret_cast<uint4 *>(tile + swz128(r, j)) = v;
}

__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 *v) {
    return make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                      pack_bf16x2(v[6], v[7]));
}

template <int LMAX>
__global__ void __launch_bounds__(TF_C, 4) k_mp_fwd_tc(EdgeGeom g, LayerIO io, int nseg, int *err) {
    using SM = FwdTcSmem<LMAX>;
    constexpr int NL = LMAX + 1, NLM = NL * NL, C = TF_C, K = TF_K;
    extern __shared__ uint8_t tf_smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_sh;
    __shared__ int wcnt[TF_C / 32];
    __shared__ __align__(16) int sJ[TF_PASS];
    __shared__ __align__(16) float4 cd[TF_PASS];   // candidate displacement and r^2
    __shared__ int cj[TF_PASS], perm[TF_PASS];
    __shared__ __align__(16) float sY[NLM][TF_PASS];
    __shared__ int err0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t raw = smem_u32(tf_smem);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *pA = tf_smem + (base - raw), *pB = pA + SM::a_bytes;
    const uint32_t sA = base, sB = base + SM::a_bytes;

    if (tid == 0) {
        mbar_init(smem_u32(&bar), 1);
        mbar_init_fence();
        err0 = *io.err;
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_sh), TF_TMEM);
    // weights of channel c = tid as row c of each l's tile
    {
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            __nv_bfloat16 hi[K], lo[K];
#pragma unroll
            for (int k = 0; k < K; ++k) split_bf16(__ldg(io.wrad + (l * K + k) * C + tid), hi[k], lo[k]);
            uint8_t *t = pA + (l >> 1) * TF_C * 128;
            const int c0 = 4 * (l & 1);
            st_chunk(t, tid, c0, pack8(hi));
            st_chunk(t, tid, c0 + 1, nseg == 3 ? pack8(lo) : z);
            st_chunk(t, tid, c0 + 2, nseg == 3 ? pack8(hi) : z);
            st_chunk(t, tid, c0 + 3, z);
        }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t idesc = idesc_bf16(TF_C, TF_CHUNK);
    uint32_t phase = 0;
    bool aborted = err0 != 0;

    for (int wi = blockIdx.x; wi < g.n_atoms && !aborted; wi += gridDim.x) {
        const int i = g.order ? __ldg(g.order + wi) : wi;
        const int rep = g.atom_rep[i];
        const float bx = g.box[3 * rep], by = g.box[3 * rep + 1], bz = g.box[3 * rep + 2];
        const float ibx = bx > 0.f ? 1.f / bx : 0.f, iby = by > 0.f ? 1.f / by : 0.f, ibz = bz > 0.f ? 1.f / bz : 0.f;
        const float xi = g.x[3 * i], yi = g.x[3 * i + 1], zi = g.x[3 * i + 2];
        const float rc2 = g.rc * g.rc;
        const int beg = g.row_ptr[i], end = g.row_ptr[i + 1];
        float2 acc[NLM];
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) acc[lm] = make_float2(0.f, 0.f);

        for (int pbeg = beg; pbeg < end && !aborted; pbeg += TF_PASS) {
            // ---- test one candidate per thread, compact the active ones
            const int e = pbeg + tid;
            bool act = false;
            if (tid < TF_PASS && e < end) {
                const int j = __ldg(g.col + e);
                const float dx = min_img(__ldg(g.x + 3 * j) - xi, bx, ibx);
                const float dy = min_img(__ldg(g.x + 3 * j + 1) - yi, by, iby);
                const float dz = min_img(__ldg(g.x + 3 * j + 2) - zi, bz, ibz);
                const float r2 = dx * dx + dy * dy + dz * dz;
                act = r2 < rc2;
                if (act) {
                    cd[tid] = make_float4(dx, dy, dz, r2);
                    cj[tid] = j;
                }
            }
            const unsigned m = __ballot_sync(DMTS_FULL, act);
            if (lane == 0) wcnt[warp] = __popc(m);
            __syncthreads();
            int off = 0, n_act = 0;
#pragma unroll
            for (int w = 0; w < TF_C / 32; ++w) {
                off += w < warp ? wcnt[w] : 0;
                n_act += wcnt[w];
            }
            const int n_pad = (n_act + TF_CHUNK - 1) / TF_CHUNK * TF_CHUNK;
            // slot of each active candidate, in candidate order
            if (act) perm[off + __popc(m & ((1u << lane) - 1u))] = tid;
            __syncthreads();
            // ---- one thread per slot: the edge's basis row, harmonics, index
            if (tid < n_act) {
                const int src = perm[tid];
                const float4 d = cd[src];
                const float r = sqrtf(d.w), inv = 1.f / r;
                float du;
                const float fc = envelope(r * g.inv_rc, g.p, &du);
                float B[K];
                bessel<K, false>(r, g.inv_rc, g.bnorm, B, nullptr);
                __nv_bfloat16 hi[K], lo[K];
#pragma unroll
                for (int k = 0; k < K; ++k) split_bf16(fc * B[k], hi[k], lo[k]);
                const uint4 h8 = pack8(hi);
                const uint4 l8 = pack8(lo), z4 = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int hh = 0; hh < (NL > 1 ? 2 : 1); ++hh) {   // the basis in both halves of the row
                    st_chunk(pB, tid, 4 * hh, h8);
                    st_chunk(pB, tid, 4 * hh + 1, h8);
                    st_chunk(pB, tid, 4 * hh + 2, l8);
                    st_chunk(pB, tid, 4 * hh + 3, z4);
                }
                float Y[NLM];
                sph<LMAX>(d.x * inv, d.y * inv, d.z * inv, Y);
#pragma unroll
                for (int lm = 0; lm < NLM; ++lm) sY[lm][tid] = Y[lm];
                sJ[tid] = cj[src];
            } else if (tid < n_pad) {
                // padding slots of the last chunk: zero basis rows and
                // harmonics, and the receiver's own (finite) features
                const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int q = 0; q < 8; ++q) st_chunk(pB, tid, q, z);
#pragma unroll
                for (int lm = 0; lm < NLM; ++lm) sY[lm][tid] = 0.f;
                sJ[tid] = i;
            }
            fence_proxy_async_smem();
            __syncthreads();

            for (int q0 = 0; q0 < n_act; q0 += TF_CHUNK) {
                if (tid == 0) {
                    tc_fence_after();
#pragma unroll
                    for (int l = 0; l < NL; ++l)
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
                            mma_bf16(tmem + l * TF_CHUNK, smem_desc(sA + (l >> 1) * TF_C * 128 + (l & 1) * 64 + kk * 32),
                                     smem_desc(sB + q0 * 128 + (l & 1) * 64 + kk * 32), idesc, kk);
                    mma_commit(smem_u32(&bar));
                }
                // neighbour features of this chunk (padding slots read the
                // receiver's own), loaded while the MMAs run
                float sj[TF_CHUNK];
#pragma unroll
                for (int u4 = 0; u4 < TF_CHUNK / 4; ++u4) {
                    const int4 jj = *reinterpret_cast<const int4 *>(&sJ[q0 + 4 * u4]);
                    sj[4 * u4] = __ldg(io.s + (size_t)jj.x * C + tid);
                    sj[4 * u4 + 1] = __ldg(io.s + (size_t)jj.y * C + tid);
                    sj[4 * u4 + 2] = __ldg(io.s + (size_t)jj.z * C + tid);
                    sj[4 * u4 + 3] = __ldg(io.s + (size_t)jj.w * C + tid);
                }
                const bool ok = mbar_wait(smem_u32(&bar), phase);
                if (!__syncthreads_and(ok ? 1 : 0)) {
                    aborted = true;
                    break;
                }
                phase ^= 1u;
                tc_fence_after();
                const int nsb = min(TF_CHUNK / 8, (n_act - q0 + 7) / 8);
#pragma unroll
                for (int b = 0; b < TF_CHUNK / 8; ++b) {
                    if (b >= nsb) break;   // uniform across the CTA
                    uint32_t rr[NL][8];
#pragma unroll
                    for (int l = 0; l < NL; ++l) tmem_ld8_issue(t_lane + l * TF_CHUNK + 8 * b, rr[l]);
                    tmem_wait_ld();
                    const int p0 = q0 + 8 * b;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float4 y[NLM];
#pragma unroll
                        for (int lm = 0; lm < NLM; ++lm) y[lm] = *reinterpret_cast<const float4 *>(&sY[lm][p0 + 4 * h]);
#pragma unroll
                        for (int pr = 0; pr < 2; ++pr) {
                            const int u = 8 * b + 4 * h + 2 * pr;   // slot within the chunk
                            const float2 s2 = make_float2(sj[u], sj[u + 1]);
#pragma unroll
                            for (int l = 0; l < NL; ++l) {
                                const int c0 = 4 * h + 2 * pr;
                                const float2 R2 = make_float2(__uint_as_float(rr[l][c0]), __uint_as_float(rr[l][c0 + 1]));
                                const float2 msg = __fmul2_rn(R2, s2);
#pragma unroll
                                for (int lm = l * l; lm < (l + 1) * (l + 1); ++lm) {
                                    const float2 y2 = pr ? make_float2(y[lm].z, y[lm].w) : make_float2(y[lm].x, y[lm].y);
                                    acc[lm] = __ffma2_rn(msg, y2, acc[lm]);
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncthreads();   // TMEM read before the next chunk's MMAs overwrite it
            }
        }
        if (aborted) break;
        // ---- receiver epilogue: A, q (and its split copy)
        float qv[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) qv[l] = 0.f;
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
            const int l = lm == 0 ? 0 : (lm < 4 ? 1 : 2);
            const float a = io.nu * (acc[lm].x + acc[lm].y);
            qv[l] = fmaf(a, a, qv[l]);
            if (io.A) io.A[((size_t)i * NLM + lm) * C + tid] = a;
        }
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            io.q[(size_t)i * NL * C + l * C + tid] = qv[l];
            if (io.q_bf16) st_split(io.q_bf16, i, NL * C, l * C + tid, qv[l]);
        }
    }

    if (aborted && tid == 0) {
        set_error(err, DMTS_E_TIMEOUT);
        mbar_wait(smem_u32(&bar), phase);   // the MMAs issued must complete before TMEM is freed
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TF_TMEM);
    }
}

template <int LMAX>
void fwd_tc_launch(const EdgeGeom &g, const LayerIO &io, int nseg, int *err, cudaStream_t st) {
    constexpr size_t smem = FwdTcSmem<LMAX>::bytes;
    static int per_sm = 0, n_sm = 0;
    if (!per_sm) {
        cudaFuncSetAttribute(k_mp_fwd_tc<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_mp_fwd_tc<LMAX>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        per_sm = resident_ctas(reinterpret_cast<const void *>(k_mp_fwd_tc<LMAX>), TF_C, smem, dev);
        // TMEM: 512 columns per SM
        per_sm = std::max(1, std::min(per_sm, 512 / TF_TMEM));
    }
    const int grid = std::min(g.n_atoms, per_sm * n_sm);
    k_mp_fwd_tc<LMAX><<<grid, TF_C, smem, st>>>(g, io, nseg, err);
    count_launch();
}

}  // namespace

int resident_ctas(const void *fn, int threads, size_t dyn_smem, int dev) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 1;
    int regs_sm = 0, smem_sm = 0, smem_blk_reserved = 0, max_thr = 0, max_blk = 0;
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_blk_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&max_thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    cudaDeviceGetAttribute(&max_blk, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    const int regs_blk = ((fa.numRegs * 32 + 255) / 256 * 256) * ((threads + 31) / 32);
    const size_t smem_blk = fa.sharedSizeBytes + dyn_smem + smem_blk_reserved;
    int n = max_blk;
    if (regs_blk > 0) n = std::min(n, regs_sm / regs_blk);
    if (smem_blk > 0) n = std::min(n, (int)(smem_sm / smem_blk));
    n = std::min(n, max_thr / threads);
    return std::max(n, 1);
}

bool mp_fwd_tc_supported(int C, int K, const LayerIO &io) { return C == TF_C && K == TF_K && !io.V; }

void launch_mp_fwd_tc(int lmax, const EdgeGeom &g, const LayerIO &io, int nseg, int *err, cudaStream_t st) {
    if (g.n_atoms == 0) return;
    if (lmax == 0) fwd_tc_launch<0>(g, io, nseg, err, st);
    else if (lmax == 1) fwd_tc_launch<1>(g, io, nseg, err, st);
    else fwd_tc_launch<2>(g, io, nseg, err, st);
}

}  // namespace dmts
