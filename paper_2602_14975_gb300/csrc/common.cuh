// Device helpers shared by the DMTS-NC kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "dmts.h"

#define DMTS_FULL 0xffffffffu

namespace dmts {

constexpr float kAccConv = 4.184e-4f;          // (kcal/mol/A)/amu -> A/fs^2
constexpr double kAccConvD = 4.184e-4;
constexpr double kBoltzmann = 8.314462618 / 4184.0;   // kcal/mol/K
constexpr double kKcalPerA3PerAtm = 101325.0 * 6.02214076e23 * 1e-30 / 4184.0;   // 1 atm in kcal/mol/A^3

// Sticky device error word (one per context).
// Host-side count of this library's kernel launches (every launch site calls
// it right after the launch); read through dmts_kernel_launches().
void count_launch();
void count_launches(unsigned long long n);   // a graph replay: the kernels its capture counted
unsigned long long launch_count();

__device__ __forceinline__ void set_error(int *err, int code) { atomicCAS(err, 0, code); }

// Row stride (floats) of the NC model's tensor-head vectors V [N][stride]:
// n_l 3-vectors padded to a multiple of four floats, so that a row is a
// whole number of 16-byte units (bulk copies).
__host__ __device__ constexpr int nc_v_stride(int n_l) { return 4 * ((3 * n_l + 3) / 4); }

// Split-bf16 operand copies of the tensor-core contractions. A logical
// [rows][K] fp32 operand is stored as bf16 [rows][2K]: column c holds
// hi = rn(v) and column K + c holds lo = rn(v - hi), so hi + lo carries
// about 16 significant bits. A contraction that accumulates hi*hi, lo*hi
// and hi*lo products in fp32 loses only the lo*lo term and the rounding of
// lo (relative ~2^-16), where a single bf16 rounding loses ~2^-9.
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}
// Element (r, c) of a split copy whose logical row length is K.
__device__ __forceinline__ void st_split(__nv_bfloat16 *base, size_t r, int K, int c, float v) {
    __nv_bfloat16 hi, lo;
    split_bf16(v, hi, lo);
    base[r * 2 * K + c] = hi;
    base[r * 2 * K + K + c] = lo;
}

// Force sums in 32.32 fixed point with 64-bit integer atomics: integer
// addition is exact and associative, so a sum does not depend on the order
// in which warps add their terms. A term must be finite and at most kFixMax
// in magnitude (2^24: up to 128 such terms fit the 64-bit sum).
constexpr float kFixScale = 4294967296.f;     // 2^32 per unit
constexpr float kFixMax = 16777216.f;
__device__ __forceinline__ bool fix_ok(float v) { return fabsf(v) < kFixMax; }   // false for NaN too
__device__ __forceinline__ long long to_fix(float v) { return __float2ll_rn(v * kFixScale); }
__device__ __forceinline__ void fix_add(unsigned long long *dst, long long q) {
    atomicAdd(dst, (unsigned long long)q);
}
__device__ __forceinline__ float fix_to_float(long long q) { return (float)((double)q * (1.0 / 4294967296.0)); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(DMTS_FULL, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(DMTS_FULL, v, o);
    return v;
}

// Replica of an atom from the replica offsets (binary search, R small).
__device__ __forceinline__ int replica_of(const int *rep_off, int n_rep, int atom) {
    int lo = 0, hi = n_rep - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(rep_off + mid) <= atom) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Minimum-image displacement on periodic axes (box > 0).
__device__ __forceinline__ float min_img(float d, float L, float invL) {
    return L > 0.f ? d - L * rintf(d * invL) : d;
}

// Polynomial envelope of Gasteiger et al. with integer exponent p, and
// its derivative with respect to u.
__device__ __forceinline__ float envelope(float u, int p, float *du) {
    if (u >= 1.f) { *du = 0.f; return 0.f; }
    float up = 1.f;
    for (int k = 0; k < p - 1; ++k) up *= u;       // u^(p-1)
    const float fp = (float)p;
    const float a = 0.5f * (fp + 1.f) * (fp + 2.f), b = fp * (fp + 2.f), c = 0.5f * fp * (fp + 1.f);
    const float upm1 = up, upw = up * u;            // u^(p-1), u^p
    const float f = 1.f - a * upw + b * upw * u - c * upw * u * u;
    *du = -a * fp * upm1 + b * (fp + 1.f) * upw - c * (fp + 2.f) * upw * u;
    return f;
}

// Bessel basis B_k(r) = sqrt(2/rc) sin(k pi r/rc)/r, k = 1..K, and dB_k/dr.
// sin(k theta), cos(k theta) from one sincospi by the Chebyshev recurrence.
template <int K, bool DERIV>
__device__ __forceinline__ void bessel(float r, float inv_rc, float norm, float *B, float *dB) {
    float s1, c1;
    sincospif(r * inv_rc, &s1, &c1);
    const float inv_r = 1.f / r;
    float sp = 0.f, s = s1, cp = 1.f, c = c1;
#pragma unroll
    for (int k = 1; k <= K; ++k) {
        B[k - 1] = norm * s * inv_r;
        if (DERIV) dB[k - 1] = norm * inv_r * ((float)k * 3.14159265358979f * inv_rc * c - s * inv_r);
        const float sn = 2.f * c1 * s - sp, cn = 2.f * c1 * c - cp;
        sp = s; s = sn; cp = c; c = cn;
    }
}

// Real spherical harmonics, component normalisation, l <= LMAX.
template <int LMAX>
__device__ __forceinline__ void sph(float x, float y, float z, float *Y) {
    Y[0] = 1.f;
    if (LMAX >= 1) {
        const float s3 = 1.7320508075688772f;
        Y[1] = s3 * x; Y[2] = s3 * y; Y[3] = s3 * z;
    }
    if (LMAX >= 2) {
        const float s15 = 3.872983346207417f, s5 = 2.23606797749979f;
        Y[4] = s15 * x * y;
        Y[5] = s15 * y * z;
        Y[6] = 0.5f * s5 * (3.f * z * z - 1.f);
        Y[7] = s15 * x * z;
        Y[8] = 0.5f * s15 * (x * x - y * y);
    }
}

// dY_lm(d/|d|)/dd = (I - n n^T) grad_n Y_lm / r, written to dY[lm*3 + a].
template <int LMAX>
__device__ __forceinline__ void sph_grad(float x, float y, float z, float inv_r, float *dY) {
    constexpr int NLM = (LMAX + 1) * (LMAX + 1);
    float g[NLM][3];
    g[0][0] = g[0][1] = g[0][2] = 0.f;
    if (LMAX >= 1) {
        const float s3 = 1.7320508075688772f;
        g[1][0] = s3; g[1][1] = 0.f; g[1][2] = 0.f;
        g[2][0] = 0.f; g[2][1] = s3; g[2][2] = 0.f;
        g[3][0] = 0.f; g[3][1] = 0.f; g[3][2] = s3;
    }
    if (LMAX >= 2) {
        const float s15 = 3.872983346207417f, s5 = 2.23606797749979f;
        g[4][0] = s15 * y; g[4][1] = s15 * x; g[4][2] = 0.f;
        g[5][0] = 0.f; g[5][1] = s15 * z; g[5][2] = s15 * y;
        g[6][0] = 0.f; g[6][1] = 0.f; g[6][2] = 3.f * s5 * z;
        g[7][0] = s15 * z; g[7][1] = 0.f; g[7][2] = s15 * x;
        g[8][0] = s15 * x; g[8][1] = -s15 * y; g[8][2] = 0.f;
    }
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) {
        const float ng = x * g[lm][0] + y * g[lm][1] + z * g[lm][2];
        dY[lm * 3 + 0] = (g[lm][0] - x * ng) * inv_r;
        dY[lm * 3 + 1] = (g[lm][1] - y * ng) * inv_r;
        dY[lm * 3 + 2] = (g[lm][2] - z * ng) * inv_r;
    }
}

__device__ __forceinline__ float silu_f(float v) { return v / (1.f + __expf(-v)); }
__device__ __forceinline__ float dsilu_f(float v) {
    const float sg = 1.f / (1.f + __expf(-v));
    return sg * (1.f + v * (1.f - sg));
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 round function
// with multipliers 0xD2511F53, 0xCD9E8D57; key bumped by the Weyl constants
// 0x9E3779B9, 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Three standard normals from one Philox block: Box-Muller on (w0, w1) and
// on (w2, w3) (second output of the latter unused); u = (w + 1/2) 2^-32.
__device__ __forceinline__ float3 gauss3(uint64_t seed, uint32_t replica, uint64_t step, uint32_t atom) {
    const uint4 w = philox4x32_10(make_uint4(atom, replica, (uint32_t)step, (uint32_t)(step >> 32)),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const float k = 2.3283064365386963e-10f;   // 2^-32
    const float u0 = fmaf((float)w.x, k, 0.5f * k), u1 = fmaf((float)w.y, k, 0.5f * k);
    const float u2 = fmaf((float)w.z, k, 0.5f * k), u3 = fmaf((float)w.w, k, 0.5f * k);
    const float r01 = sqrtf(-2.f * logf(u0)), r23 = sqrtf(-2.f * logf(u2));
    float s1, c1, s3, c3;
    sincospif(2.f * u1, &s1, &c1);
    sincospif(2.f * u3, &s3, &c3);
    (void)s3;
    return make_float3(r01 * c1, r01 * s1, r23 * c3);
}

}  // namespace dmts
