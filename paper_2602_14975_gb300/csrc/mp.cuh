// Kernels of the message-passing layer (edge embedding + segmented
// scatter-sum) and of its adjoint, plus the node-level GEMMs of the MLPs.
#pragma once
#include "common.cuh"

namespace dmts {

// Geometry shared by the edge kernels of one model evaluation.
struct EdgeGeom {
    const float *x;          // [N][3]
    const int *atom_rep;     // [N] replica of each atom
    const float *box;        // [R][3]
    const int *row_ptr;      // [N+1] stored list (cutoff + skin)
    const int *col;
    int n_atoms;
    float rc, inv_rc, bnorm; // model cutoff, 1/rc, sqrt(2/rc)
    int p;                   // envelope exponent
    const int *order;        // nullable: atoms in processing order (cell order), else identity
};

// Node-level arrays for one layer.
struct LayerIO {
    const float *s;          // [N][C] input features s^t
    const float *wrad;       // [L+1][K][C]
    float nu;
    float *A;                // [N][NLM][C]  (forward out; nullable: not stored)
    float *q;                // [N][(LMAX+1)C] (forward out, fp32)
    __nv_bfloat16 *q_bf16;   // optional split-bf16 copy of q, [N][2(LMAX+1)C] (forward out)
    const float *U;          // optional: tensor-head mix U[n_l][C] (NC embedding)
    float *V;                // optional: V[N][nc_v_stride(n_l)], V[i][3h + a] = sum_c U[h][c] A[1+a][c]
    int n_l;
    const float *gA;         // [N][NLM][C]  (backward in)
    const float *gs_in;      // [N][C]       (backward in)
    float *gs_out;           // [N][C]       (backward out; nullable: not computed)
    __nv_bfloat16 *gs_out_bf16;  // optional split-bf16 copy of gs_out, [N][2C]
    unsigned long long *Ffix;  // [N][3] (backward): forces added in 32.32 fixed point
    unsigned long long *Wfix;  // [N] (backward, nullable): per-atom virial proxy, pair form, fixed point
    int *err;
};

template <int CPW>
struct VecF;
template <> struct VecF<1> { using T = float; };
template <> struct VecF<2> { using T = float2; };
template <> struct VecF<4> { using T = float4; };

template <int CPW>
__device__ __forceinline__ void ldv(const float *p, float *v) {
    if constexpr (CPW == 4) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (CPW == 2) {
        float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = t.x; v[1] = t.y;
    } else {
        v[0] = __ldg(p);
    }
}

template <int CPW>
__device__ __forceinline__ void stv(float *p, const float *v) {
    if constexpr (CPW == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (CPW == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
        *p = v[0];
    }
}

void launch_mp_fwd(int C, int lmax, int K, const EdgeGeom &g, const LayerIO &io, cudaStream_t st);
// The forward layer with the radial contraction R = W B on the tensor cores
// (split-bf16 operands, nseg as for launch_gemm_tc): C = 128, K = 8 and no
// tensor-head output (io.V null) only; err receives DMTS_E_TIMEOUT if a
// bounded wait on the tensor cores runs out.
bool mp_fwd_tc_supported(int C, int K, const LayerIO &io);
void launch_mp_fwd_tc(int lmax, const EdgeGeom &g, const LayerIO &io, int nseg, int *err, cudaStream_t st);
void launch_mp_bwd(int C, int lmax, int K, const EdgeGeom &g, const LayerIO &io, cudaStream_t st);
// The adjoint's fixed-point forces (and virial, Wfix nullable) -> fp32 F and
// W, the fixed-point words cleared for the next evaluation.
void launch_fix_convert(int n, unsigned long long *Ffix, float *F, unsigned long long *Wfix, float *W, cudaStream_t st);

// CTAs of a kernel resident per SM, from its register and shared-memory use
// and the device's limits (the largest shared-memory carveout).
int resident_ctas(const void *fn, int threads, size_t dyn_smem, int dev);

// ---------------------------------------------------------------- GEMM ----
enum EpiMode {
    EPI_STORE = 0,           // out = v
    EPI_BIAS_SILU = 1,       // H = v + bias; out = silu(H) (out, H and the bf16 copy each nullable)
    EPI_RESID = 2,           // out = res + v + bias
    EPI_DSILU = 3,           // out = v * dsilu(H)
    EPI_GA = 4,              // gA[m][lm][c] = 2 A[m][lm][c] v,  n = l*C + c
    EPI_READOUT = 5,         // z = v + bias: out = wo silu(z), out2 = scale wo dsilu(z)
};

struct Epi {
    int mode;
    float *out;
    __nv_bfloat16 *out_bf16;   // optional split-bf16 copy of out, [M][2N] (hi | lo)
    float *out2;
    const float *bias;
    const float *res;          // residual input [M][N]
    float *H;                  // pre-activation store (nullable) / load
    const float *A;            // EPI_GA
    const float *wo;           // EPI_READOUT
    float scale;
    int C, lmax;               // EPI_GA
};

// Out[M][N] = Act[M][K] x op(W) where op(W) = W^T for W [N][K] (trans = 1)
// or W for W [K][N] (trans = 0); fp32 SIMT.
void launch_gemm_f32(int M, int N, int K, const float *Act, const float *W, int trans, const Epi &e,
                     cudaStream_t st);
// Out[M][N] = Act[M][K] x Wt^T on the tensor cores (tcgen05, bf16 operands,
// fp32 accumulator in tensor memory), Wt K-major [N][K]. With split = 1 both
// operands are split-bf16 copies (rows of 2K: hi | lo, common.cuh) and
// nseg = 3 accumulates hi*hi + lo*hi + hi*lo (nseg = 1: hi*hi only); with
// split = 0 they are plain bf16 [M][K] / [N][K] and nseg must be 1. Needs
// K % 64 == 0, N % 16 == 0, M >= 1 (rows past M of the last 128-row tile
// read as zeros and are not stored) and 16-byte aligned operands; returns 0
// when launched, < 0 when the shape is not supported.
int launch_gemm_tc(int M, int N, int K, const __nv_bfloat16 *Act, const __nv_bfloat16 *Wt, const Epi &e, int *err,
                   cudaStream_t st, int split, int nseg);
bool gemm_tc_supported(int N, int K);

// Per-replica FP64 sums of per-atom values: out[r] = sum_{i in r} v[i].
void launch_replica_sum(const float *v, const int *rep_off, int n_rep, double *out, int accumulate,
                        cudaStream_t st);

}  // namespace dmts
