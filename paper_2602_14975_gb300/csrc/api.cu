// Host side of the C ABI: context, device models, workspace, force
// evaluations, the Algorithm-1 driver (respa_step) and host helpers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "engine.cuh"
#include "ptx.cuh"

using namespace dmts;

// ------------------------------------------------------------ utilities --
namespace dmts {

static thread_local std::string g_tls_error;

bool ck(dmts_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    if (ctx) ctx->last_error = buf;
    g_tls_error = buf;
    return false;
}

dmts_status fail(dmts_ctx *ctx, dmts_status s, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    g_tls_error = msg;
    return s;
}

static std::atomic<unsigned long long> g_alloc_gen{0};
unsigned long long alloc_generation() { return g_alloc_gen.load(std::memory_order_relaxed); }
void bump_alloc_generation() { g_alloc_gen.fetch_add(1, std::memory_order_relaxed); }

bool Buf::ensure(size_t bytes) {
    if (bytes <= cap) return true;
    bump_alloc_generation();
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max<size_t>(bytes, 256);
    if (cudaMalloc(&p, want) != cudaSuccess) {
        p = nullptr;
        return false;
    }
    cap = want;
    return true;
}

// ensure() for a buffer that must hold zeros whenever it is not in use: a
// new allocation is cleared on the stream.
static bool ensure_zeroed(dmts_ctx *ctx, Buf &b, size_t bytes, cudaStream_t st) {
    if (bytes <= b.cap) return true;
    if (!b.ensure(bytes)) return false;
    return ck(ctx, cudaMemsetAsync(b.p, 0, b.cap, st), "workspace clear");
}

void Buf::release() {
    if (p) {
        bump_alloc_generation();
        cudaFree(p);
    }
    p = nullptr;
    cap = 0;
}

// float -> bf16 bits, round to nearest even (NaN kept quiet)
static uint16_t bf16_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static bool upload(DevModel &m, const std::vector<float> &h) {
    bump_alloc_generation();
    if (cudaMalloc(&m.dev, h.size() * sizeof(float)) != cudaSuccess) return false;
    return cudaMemcpy(m.dev, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
}

static dmts_status load_model(dmts_ctx *ctx, const dmts_model *in, bool is_nc, DevModel &m) {
    m.L = is_nc ? 1 : in->L;
    m.C = in->C;
    m.lmax = is_nc ? 1 : in->lmax;
    m.K = in->K;
    m.S = in->n_species;
    m.nc = in->n_c;
    m.nl = in->n_l;
    m.rc = in->rc;
    m.p = (int)lrintf(in->p_env);
    m.nu = in->nu;
    m.scale = in->scale;
    if (in->precision != DMTS_FP32 && in->precision != DMTS_BF16 && in->precision != DMTS_BF16_PLAIN)
        return fail(ctx, DMTS_E_INVALID, "precision must be DMTS_FP32, DMTS_BF16 or DMTS_BF16_PLAIN");
    m.bf16 = in->precision != DMTS_FP32;
    m.nseg = in->precision == DMTS_BF16 ? 3 : 1;
    const int C = m.C, K = m.K, NL = m.lmax + 1, S = m.S;
    if (K != 8) return fail(ctx, DMTS_E_INVALID, "only K = 8 Bessel functions are supported");
    if (!(C == 32 || C == 64 || C == 128)) return fail(ctx, DMTS_E_INVALID, "C must be 32, 64 or 128");
    if (m.lmax < 0 || m.lmax > 2) return fail(ctx, DMTS_E_INVALID, "lmax must be 0..2");
    if (m.L < 1 || m.L > DMTS_MAX_LAYERS) return fail(ctx, DMTS_E_INVALID, "bad layer count");
    if (S < 1 || S > DMTS_MAX_SPECIES) return fail(ctx, DMTS_E_INVALID, "bad species count");
    if (m.p < 2 || m.p > 12 || std::fabs(in->p_env - (float)m.p) > 1e-6f)
        return fail(ctx, DMTS_E_INVALID, "p_env must be an integer in 2..12");
    if (!(m.rc > 0.f)) return fail(ctx, DMTS_E_INVALID, "rc must be positive");
    if (is_nc && (C > 64 || m.nc != 8 || m.nl < 1 || m.nl > 4))
        return fail(ctx, DMTS_E_INVALID, "NC model: C <= 64, n_c = 8, 1 <= n_l <= 4");
    if (m.bf16 && (C < 64 || (is_nc && C != 64)))
        return fail(ctx, DMTS_E_INVALID, "bf16 MLP contractions need C >= 64 (K-chunks of 64)");
    long long expect;
    if (!is_nc)
        expect = (long long)S * C + (long long)m.L * (NL * K * C + NL * C * C + C + C * C + C) + C * C + 2 * C;
    else {
        const int H = K + m.nl;
        expect = (long long)S * C + 2 * K * C + 2 * C * C + C + C * C + C + m.nl * C + 2LL * H * m.nc * C;
    }
    if (in->n_weights != expect || !in->weights)
        return fail(ctx, DMTS_E_INVALID, "weight blob size does not match the model sizes");
    std::vector<float> h(in->weights, in->weights + expect);
    if (!upload(m, h)) return fail(ctx, DMTS_E_OOM, "weight upload failed");
    m.n_weights = (size_t)expect;
    // offsets (same order as the blob)
    size_t o = 0;
    auto take = [&](size_t n) { float *p = m.dev + o; o += n; return p; };
    m.emb = take((size_t)S * C);
    for (int t = 0; t < m.L; ++t) {
        m.wrad[t] = take((size_t)NL * K * C);
        m.w1[t] = take((size_t)C * NL * C);
        m.b1[t] = take(C);
        m.w2[t] = take((size_t)C * C);
        m.b2[t] = take(C);
    }
    if (!is_nc) {
        m.wr = take((size_t)C * C);
        m.br = take(C);
        m.wo = take(C);
    } else {
        const int H = K + m.nl;
        m.U = take((size_t)m.nl * C);
        m.Wqk = take((size_t)2 * H * m.nc * C);   // Wq rows then Wk rows: one [2 H n_c][C] matrix
    }
    if (m.bf16) {
        // split-bf16 host copies, K-major: each output row of the logical
        // [rows'][K'] matrix holds hi = rn(w) in columns [0, K') and
        // lo = rn(w - hi) in [K', 2K') (round to nearest even)
        std::vector<uint16_t> hb;
        auto off_of = [&](const float *p) { return (size_t)(p - m.dev); };
        auto push = [&](const float *p, int rows, int cols, bool transpose) {
            const size_t start = hb.size();
            const float *src = h.data() + off_of(p);
            hb.resize(start + (size_t)2 * rows * cols);
            const int kk = transpose ? rows : cols;   // logical row length of the copy
            for (int r = 0; r < rows; ++r)
                for (int c = 0; c < cols; ++c) {
                    const float v = src[(size_t)r * cols + c];
                    const uint16_t hi = bf16_bits(v);
                    const uint32_t hu = (uint32_t)hi << 16;
                    float hf;
                    memcpy(&hf, &hu, 4);
                    const uint16_t lo = bf16_bits(v - hf);
                    const size_t orow = transpose ? (size_t)c : (size_t)r, ocol = transpose ? (size_t)r : (size_t)c;
                    hb[start + orow * 2 * kk + ocol] = hi;
                    hb[start + orow * 2 * kk + kk + ocol] = lo;
                }
            return start;
        };
        std::vector<size_t> o_w1(m.L), o_w2(m.L), o_w1t(m.L), o_w2t(m.L);
        for (int t = 0; t < m.L; ++t) {
            o_w1[t] = push(m.w1[t], C, NL * C, false);
            o_w2[t] = push(m.w2[t], C, C, false);
            o_w1t[t] = push(m.w1[t], C, NL * C, true);
            o_w2t[t] = push(m.w2[t], C, C, true);
        }
        size_t o_wr = 0, o_wrt = 0, o_qk = 0;
        if (!is_nc) {
            o_wr = push(m.wr, C, C, false);
            o_wrt = push(m.wr, C, C, true);
        } else {
            o_qk = push(m.Wqk, 2 * (K + m.nl) * m.nc, C, false);
        }
        bump_alloc_generation();
        if (cudaMalloc(&m.dev_bf, hb.size() * 2) != cudaSuccess ||
            cudaMemcpy(m.dev_bf, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(ctx, DMTS_E_OOM, "bf16 weight upload failed");
        for (int t = 0; t < m.L; ++t) {
            m.w1_bf[t] = m.dev_bf + o_w1[t];
            m.w2_bf[t] = m.dev_bf + o_w2[t];
            m.w1t_bf[t] = m.dev_bf + o_w1t[t];
            m.w2t_bf[t] = m.dev_bf + o_w2t[t];
        }
        if (!is_nc) {
            m.wr_bf = m.dev_bf + o_wr;
            m.wrt_bf = m.dev_bf + o_wrt;
        } else {
            m.wqk_bf = m.dev_bf + o_qk;
        }
    }
    return DMTS_OK;
}

// Species-pair table of the screened repulsion (host FP64 -> float).
RepTable rep_table(const dmts_ctx *ctx) {
    static const double Z[5] = {1.0, 6.0, 7.0, 8.0, 16.0};
    RepTable t;
    memset(&t, 0, sizeof t);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            t.zz[i][j] = (float)(332.0637133 * Z[i] * Z[j]);
            t.inv_a[i][j] = (float)((std::pow(Z[i], 0.23) + std::pow(Z[j], 0.23)) / (0.8854 * 0.529177210903));
        }
    t.rc = ctx->prior.rep_rc;
    t.inv_rc = t.rc > 0.f ? 1.f / t.rc : 0.f;
    t.p = (int)lrintf(ctx->prior.rep_p);
    t.on = t.rc > 0.f;
    return t;
}

// -------------------------------------------------------- force pieces --
EdgeGeom edge_geom(const SysView &s, const int *row_ptr, const int *col, const DevModel &m) {
    EdgeGeom g;
    g.order = s.order;
    g.x = s.x;
    g.atom_rep = s.atom_rep;
    g.box = s.box;
    g.row_ptr = row_ptr;
    g.col = col;
    g.n_atoms = s.n;
    g.rc = m.rc;
    g.inv_rc = 1.f / m.rc;
    g.bnorm = sqrtf(2.f / m.rc);
    g.p = m.p;
    return g;
}

static Epi epi(int mode) {
    Epi e;
    memset(&e, 0, sizeof e);
    e.mode = mode;
    return e;
}

// One node-level contraction: the tensor cores (split-bf16 operands) for a
// model that runs its MLPs in bf16, whatever the number of rows M (a batch
// smaller than one 128-row tile reads zero-filled rows), so that an atom's
// arithmetic never depends on the batch it is in; the fp32 SIMT kernel for
// an fp32 model. trans/W32 describe the fp32 weight, Wt16 the K-major
// split-bf16 copy. False (with the context's error text set) when a bf16
// model's contraction cannot be launched.
static bool contract(dmts_ctx *ctx, const DevModel &m, int M, int N, int K, const float *A32,
                     const __nv_bfloat16 *A16, const float *W32, int trans, const __nv_bfloat16 *Wt16, const Epi &e,
                     cudaStream_t st, const char *tag_tc, const char *tag_f32) {
    if (m.bf16) {
        ProfScope ps(ctx, tag_tc, st);
        if (A16 && Wt16 && launch_gemm_tc(M, N, K, A16, Wt16, e, ctx->d_err, st, 1, m.nseg) == 0) return true;
        fail(ctx, DMTS_E_CUDA, "tensor-core contraction could not be launched (operands or tensor map)");
        return false;
    }
    ProfScope ps(ctx, tag_f32, st);
    launch_gemm_f32(M, N, K, A32, W32, trans, e, st);
    return true;
}

// U_MP (+ prior) and F = -grad U for a batch.
dmts_status cons_eval(dmts_ctx *ctx, const SysView &s, const int *row_ptr, const int *col, double *energy,
                      float *forces, int flags, cudaStream_t st, double *virial) {
    const DevModel &m = ctx->cons;
    const int N = s.n, C = m.C, L = m.L, NL = m.lmax + 1, NLM = NL * NL;
    Workspace &w = ctx->ws;
    const size_t nc_ = (size_t)N * C;
    const bool bf = m.bf16;
    if (!w.s.ensure(sizeof(float) * nc_ * (L + 1)) || !w.A.ensure(sizeof(float) * nc_ * NLM * L) ||
        !w.q.ensure(sizeof(float) * nc_ * NL) || !w.h.ensure(sizeof(float) * nc_ * L) ||
        !w.act.ensure(sizeof(float) * nc_) || !w.u.ensure(sizeof(float) * nc_) || !w.gz.ensure(sizeof(float) * nc_) ||
        !w.gs0.ensure(sizeof(float) * nc_) || !w.gs1.ensure(sizeof(float) * nc_) ||
        !w.gA.ensure(sizeof(float) * nc_ * NLM) || !w.e_atom.ensure(sizeof(float) * (N + 1)) ||
        !w.ftmp.ensure(sizeof(float) * 3 * (N + 1)) || (virial && !w.cons_w.ensure(sizeof(float) * (N + 1))) ||
        (forces && !ensure_zeroed(ctx, w.cons_ffix, sizeof(unsigned long long) * 3 * (N + 1), st)) ||
        (forces && virial && !ensure_zeroed(ctx, w.cons_wfix, sizeof(unsigned long long) * (N + 1), st)))
        return fail(ctx, DMTS_E_OOM, "workspace allocation failed");
    // split-bf16 copies: 4 bytes per logical element (hi and lo)
    if (bf && (!w.q_bf.ensure(4 * nc_ * NL + 16) || !w.act_bf.ensure(4 * nc_ + 16) || !w.s_bf.ensure(4 * nc_ + 16) ||
               !w.gz_bf.ensure(4 * nc_ + 16) || !w.gs0_bf.ensure(4 * nc_ + 16) || !w.gs1_bf.ensure(4 * nc_ + 16)))
        return fail(ctx, DMTS_E_OOM, "workspace allocation failed");
    float *S = (float *)w.s.p, *A = (float *)w.A.p, *q = (float *)w.q.p, *H = (float *)w.h.p;
    float *act = (float *)w.act.p, *u = (float *)w.u.p, *gz = (float *)w.gz.p;
    float *gs0 = (float *)w.gs0.p, *gs1 = (float *)w.gs1.p, *gA = (float *)w.gA.p;
    float *e_atom = (float *)w.e_atom.p;
    __nv_bfloat16 *q_bf = bf ? (__nv_bfloat16 *)w.q_bf.p : nullptr, *act_bf = bf ? (__nv_bfloat16 *)w.act_bf.p : nullptr;
    __nv_bfloat16 *s_bf = bf ? (__nv_bfloat16 *)w.s_bf.p : nullptr, *gz_bf = bf ? (__nv_bfloat16 *)w.gz_bf.p : nullptr;
    __nv_bfloat16 *gs0_bf = bf ? (__nv_bfloat16 *)w.gs0_bf.p : nullptr, *gs1_bf = bf ? (__nv_bfloat16 *)w.gs1_bf.p : nullptr;
    const EdgeGeom g = edge_geom(s, row_ptr, col, m);
    if (!(flags & kFlagEmbedded)) { ProfScope ps(ctx, "embed", st); launch_embed(N, C, s.species, m.emb, S, st); }
    for (int t = 0; t < L; ++t) {
        LayerIO io;
        memset(&io, 0, sizeof io);
        io.s = S + nc_ * t;
        io.wrad = m.wrad[t];
        io.nu = m.nu;
        io.A = A + nc_ * NLM * t;
        io.q = q;
        io.q_bf16 = q_bf;
        io.err = ctx->d_err;
        {
            ProfScope ps(ctx, "mp_fwd", st);
            if (bf && mp_fwd_tc_supported(C, m.K, io)) launch_mp_fwd_tc(m.lmax, g, io, m.nseg, ctx->d_err, st);
            else launch_mp_fwd(C, m.lmax, m.K, g, io, st);
        }
        Epi e1 = epi(EPI_BIAS_SILU);
        e1.bias = m.b1[t];
        e1.H = H + nc_ * t;
        e1.out = bf ? nullptr : act;            // the tensor-core path reads only the split-bf16 copy
        e1.out_bf16 = act_bf;
        if (!contract(ctx, m, N, C, NL * C, q, q_bf, m.w1[t], 1, m.w1_bf[t], e1, st, "gemm_tc", "gemm"))
            return DMTS_E_CUDA;
        Epi e2 = epi(EPI_RESID);
        e2.bias = m.b2[t];
        e2.res = S + nc_ * t;
        e2.out = S + nc_ * (t + 1);
        e2.out_bf16 = t == L - 1 ? s_bf : nullptr;
        if (!contract(ctx, m, N, C, C, act, act_bf, m.w2[t], 1, m.w2_bf[t], e2, st, "gemm_tc", "gemm"))
            return DMTS_E_CUDA;
    }
    Epi er = epi(EPI_READOUT);
    er.bias = m.br;
    er.wo = m.wo;
    er.scale = m.scale;
    er.out = u;
    er.out2 = gz;
    er.out_bf16 = gz_bf;
    if (!contract(ctx, m, N, C, C, S + nc_ * L, s_bf, m.wr, 1, m.wr_bf, er, st, "gemm_tc", "gemm"))
        return DMTS_E_CUDA;
    { ProfScope ps(ctx, "rowsum", st); launch_rowsum(N, C, u, m.scale, e_atom, st); }
    if (forces) {
        // dU/ds^L = gz Wr
        Epi eg = epi(EPI_STORE);
        eg.out = gs0;
        eg.out_bf16 = gs0_bf;
        if (!contract(ctx, m, N, C, C, gz, gz_bf, m.wr, 0, m.wrt_bf, eg, st, "gemm_tc", "gemm"))
            return DMTS_E_CUDA;
        float *gin = gs0, *gout = gs1;
        __nv_bfloat16 *gin_bf = gs0_bf, *gout_bf = gs1_bf;
        for (int t = L - 1; t >= 0; --t) {
            Epi ed = epi(EPI_DSILU);
            ed.H = H + nc_ * t;
            ed.out = act;                       // g_h
            ed.out_bf16 = act_bf;
            if (!contract(ctx, m, N, C, C, gin, gin_bf, m.w2[t], 0, m.w2t_bf[t], ed, st, "gemm_tc", "gemm"))
                return DMTS_E_CUDA;
            Epi ea = epi(EPI_GA);
            ea.A = A + nc_ * NLM * t;
            ea.out = gA;
            ea.C = C;
            ea.lmax = m.lmax;
            if (!contract(ctx, m, N, NL * C, C, act, act_bf, m.w1[t], 0, m.w1t_bf[t], ea, st, "gemm_tc", "gemm"))
                return DMTS_E_CUDA;
            LayerIO io;
            memset(&io, 0, sizeof io);
            io.s = S + nc_ * t;
            io.wrad = m.wrad[t];
            io.nu = m.nu;
            io.gA = gA;
            io.gs_in = gin;
            io.gs_out = t > 0 ? gout : nullptr;   // layer 0's inputs are the species embedding
            io.gs_out_bf16 = t > 0 ? gout_bf : nullptr;
            io.Ffix = (unsigned long long *)w.cons_ffix.p;
            io.Wfix = virial ? (unsigned long long *)w.cons_wfix.p : nullptr;
            io.err = ctx->d_err;
            { ProfScope ps(ctx, "mp_bwd", st); launch_mp_bwd(C, m.lmax, m.K, g, io, st); }
            std::swap(gin, gout);
            std::swap(gin_bf, gout_bf);
        }
        // the layers' fixed-point sums -> F (and the virial), cleared
        ProfScope ps(ctx, "fix_convert", st);
        launch_fix_convert(N, (unsigned long long *)w.cons_ffix.p, forces,
                           virial ? (unsigned long long *)w.cons_wfix.p : nullptr,
                           virial ? (float *)w.cons_w.p : nullptr, st);
    }
    if (flags & DMTS_WITH_PRIOR) {
        PriorArgs pa;
        pa.x = s.x;
        pa.atom_rep = s.atom_rep;
        pa.box = s.box;
        pa.row_ptr = row_ptr;
        pa.col = col;
        pa.species = s.species;
        pa.mol_id = s.mol_id;
        pa.n_atoms = N;
        pa.lj_eps = ctx->prior.lj_eps;
        pa.lj_sigma = ctx->prior.lj_sigma;
        pa.lj_rc = ctx->prior.lj_rc;
        pa.lj_p = (int)lrintf(ctx->prior.lj_p);
        pa.bonds = {s.bond_ptr, s.bond_idx, s.bond_r0, ctx->prior.k_bond};
        pa.rep = rep_table(ctx);
        pa.F = forces ? forces : (float *)w.ftmp.p;
        if (!forces) cudaMemsetAsync(w.ftmp.p, 0, sizeof(float) * 3 * N, st);
        pa.e_atom = e_atom;
        pa.W = virial ? (float *)w.cons_w.p : nullptr;
        pa.order = s.order;
        pa.err = ctx->d_err;
        { ProfScope ps(ctx, "prior", st); launch_prior(pa, st); }
    }
    if (energy) { ProfScope ps(ctx, "replica_sum", st); launch_replica_sum(e_atom, s.rep_off, s.n_rep, energy, 0, st); }
    if (virial) {
        ProfScope ps(ctx, "replica_sum", st);
        launch_replica_sum((const float *)w.cons_w.p, s.rep_off, s.n_rep, virial, 0, st);
    }
    return DMTS_OK;
}

// F_NC (+ bonds, F_rep), mean-subtracted; net = per-replica sum before subtraction.
dmts_status nc_eval(dmts_ctx *ctx, const SysView &s, const int *row_ptr, const int *col, float *forces,
                    double *net, int flags, cudaStream_t st, double *virial, int virial_accumulate) {
    const DevModel &m = ctx->nc;
    const int N = s.n, C = m.C, H = m.K + m.nl, QKW = 2 * H * m.nc;
    Workspace &w = ctx->ws;
    const size_t nc_ = (size_t)N * C;
    const bool bf = m.bf16;
    if (!w.nc_s.ensure(sizeof(float) * nc_ * 2) ||
        !w.nc_q.ensure(sizeof(float) * nc_ * 2) ||
        !w.nc_act.ensure(sizeof(float) * nc_) || !w.nc_qk.ensure(sizeof(float) * (size_t)N * QKW) ||
        !w.nc_v.ensure(sizeof(float) * (size_t)N * nc_v_stride(m.nl)) || !w.nc_f.ensure(sizeof(float) * 3 * (N + 1)) ||
        !ensure_zeroed(ctx, w.nc_ffix, sizeof(unsigned long long) * 3 * (N + 1), st) ||
        !ensure_zeroed(ctx, w.nc_next, sizeof(unsigned), st) ||
        !w.nc_sum.ensure(sizeof(unsigned long long) * 3 * (s.n_rep + 1)) ||
        !w.ms_scratch.ensure(mean_sub_scratch_bytes(N, s.n_rep)) ||
        (virial && !w.nc_w.ensure(sizeof(float) * (N + 1))))
        return fail(ctx, DMTS_E_OOM, "workspace allocation failed");
    if (bf && (!w.nc_q_bf.ensure(4 * nc_ * 2 + 16) || !w.nc_act_bf.ensure(4 * nc_ + 16) || !w.nc_s_bf.ensure(4 * nc_ + 16)))
        return fail(ctx, DMTS_E_OOM, "workspace allocation failed");
    __nv_bfloat16 *q_bf = bf ? (__nv_bfloat16 *)w.nc_q_bf.p : nullptr;
    __nv_bfloat16 *act_bf = bf ? (__nv_bfloat16 *)w.nc_act_bf.p : nullptr;
    __nv_bfloat16 *s_bf = bf ? (__nv_bfloat16 *)w.nc_s_bf.p : nullptr;
    float *s0 = (float *)w.nc_s.p, *s1 = s0 + nc_;
    const EdgeGeom g = edge_geom(s, row_ptr, col, m);
    if (!(flags & kFlagEmbedded)) { ProfScope ps(ctx, "embed", st); launch_embed(N, C, s.species, m.emb, s0, st); }
    LayerIO io;
    memset(&io, 0, sizeof io);
    io.s = s0;
    io.wrad = m.wrad[0];
    io.nu = m.nu;
    io.A = (flags & kFlagKeepPre) ? (float *)w.dist_A.p : nullptr;   // the head needs q and V only; kept for the distillation
    io.q = (float *)w.nc_q.p;
    io.q_bf16 = q_bf;
    io.U = m.U;
    io.V = (float *)w.nc_v.p;
    io.n_l = m.nl;
    io.err = ctx->d_err;
    { ProfScope ps(ctx, "nc_mp_fwd", st); launch_mp_fwd(C, 1, m.K, g, io, st); }
    Epi e1 = epi(EPI_BIAS_SILU);
    e1.bias = m.b1[0];
    e1.H = (flags & kFlagKeepPre) ? (float *)w.dist_h.p : nullptr;   // kept only for the distillation
    // the tensor-core path reads only the split-bf16 copy; the distillation's
    // weight gradient reads the fp32 activation
    e1.out = (bf && !(flags & kFlagKeepPre)) ? nullptr : (float *)w.nc_act.p;
    e1.out_bf16 = act_bf;
    if (!contract(ctx, m, N, C, 2 * C, io.q, q_bf, m.w1[0], 1, m.w1_bf[0], e1, st, "nc_gemm_tc", "nc_gemm"))
        return DMTS_E_CUDA;
    Epi e2 = epi(EPI_RESID);
    e2.bias = m.b2[0];
    e2.res = s0;
    e2.out = s1;
    e2.out_bf16 = s_bf;
    if (!contract(ctx, m, N, C, C, (float *)w.nc_act.p, act_bf, m.w2[0], 1, m.w2_bf[0], e2, st, "nc_gemm_tc", "nc_gemm"))
        return DMTS_E_CUDA;
    Epi e3 = epi(EPI_STORE);
    e3.out = (float *)w.nc_qk.p;
    if (!contract(ctx, m, N, QKW, C, s1, s_bf, m.Wqk, 1, m.wqk_bf, e3, st, "nc_gemm_tc", "nc_gemm"))
        return DMTS_E_CUDA;
    NCHeadArgs a;
    a.x = s.x;
    a.atom_rep = s.atom_rep;
    a.box = s.box;
    a.row_ptr = row_ptr;
    a.col = col;
    a.n_atoms = N;
    a.rc = m.rc;
    a.inv_rc = 1.f / m.rc;
    a.bnorm = sqrtf(2.f / m.rc);
    a.p = m.p;
    a.QK = (float *)w.nc_qk.p;
    a.V = (float *)w.nc_v.p;
    a.scale = m.scale;
    a.bonds = {nullptr, nullptr, nullptr, 0.f};
    if (flags & DMTS_WITH_BONDS) a.bonds = {s.bond_ptr, s.bond_idx, s.bond_r0, ctx->prior.k_bond};
    a.rep = rep_table(ctx);
    a.species = s.species;
    a.Ffix = (unsigned long long *)w.nc_ffix.p;
    a.sum = (unsigned long long *)w.nc_sum.p;
    a.next = (unsigned *)w.nc_next.p;
    a.n_rep = s.n_rep;
    a.W = virial ? (float *)w.nc_w.p : nullptr;
    a.order = s.order;
    a.err = ctx->d_err;
    { ProfScope ps(ctx, "nc_head", st); launch_nc_head(m.K, m.nc, m.nl, a, st); }
    if (N == 0 && !ck(ctx, cudaMemsetAsync(w.nc_sum.p, 0, sizeof(unsigned long long) * 3 * s.n_rep, st), "sums"))
        return DMTS_E_CUDA;   // no head launch clears them
    {
        // fp32 forces and the replicas' exact sums; the mean subtraction here
        // or, inside respa_step, in the next integrator launch
        ProfScope ps(ctx, "mean_sub", st);
        launch_nc_convert(N, s.atom_rep, a.Ffix, (float *)w.nc_f.p, a.sum, a.next, st);
        if (!(flags & kFlagDeferMean))
            launch_nc_apply(N, s.atom_rep, s.rep_off, s.n_rep, (float *)w.nc_f.p, forces, a.sum, net, ctx->d_err, st);
    }
    if (virial) {
        ProfScope ps(ctx, "replica_sum", st);
        launch_replica_sum((const float *)w.nc_w.p, s.rep_off, s.n_rep, virial, virial_accumulate, st);
    }
    return DMTS_OK;
}

__global__ void k_set_int(int *p, int v) { *p = v; }

// Rebuilds the state's lists now, for its current positions (after the
// positions were replaced, e.g. by a saved frame).
void state_force_rebuild(dmts_ctx *ctx, dmts_state *stt, cudaStream_t st) {
    StateInternal *si = (StateInternal *)stt->internal;
    if (!si) return;
    k_set_int<<<1, 1, 0, st>>>((int *)si->gate.p, 1);
    count_launch();
    rebuild_lists(ctx, si, state_view(stt), st);
}

// Host-side grid set-up for every replica (box and offsets copied to host).
dmts_status setup_grids(dmts_ctx *ctx, const std::vector<int> &rep_off, const std::vector<float> &box,
                        float r_list, std::vector<CellGrid> &grids, int &n_cells, float grid_margin) {
    const int R = (int)rep_off.size() - 1;
    grids.resize(R);
    n_cells = 0;
    for (int r = 0; r < R; ++r) {
        CellGrid g;
        memset(&g, 0, sizeof g);
        const bool periodic = box[3 * r] > 0.f;
        for (int a = 0; a < 3; ++a) {
            const float L = box[3 * r + a];
            if (periodic != (L > 0.f)) return fail(ctx, DMTS_E_INVALID, "box must be periodic on all axes or none");
            if (periodic) {
                if (!(r_list < 0.5f * L)) return fail(ctx, DMTS_E_INVALID, "list cutoff must be < box/2");
                g.box[a] = L;
                g.dim[a] = std::max(1, std::min(64, (int)std::floor(L / (r_list * (1.f + grid_margin)))));
                g.org[a] = 0.f;
                g.inv_h[a] = (float)g.dim[a] / L;
            } else {
                const int nr = rep_off[r + 1] - rep_off[r];
                g.dim[a] = std::max(1, std::min(32, (int)std::lround(std::cbrt(nr / 8.0))));
                g.inv_h[a] = 1.f / r_list;
            }
        }
        g.cell_off = n_cells;
        n_cells += g.dim[0] * g.dim[1] * g.dim[2];
        grids[r] = g;
    }
    return DMTS_OK;
}


SysView state_view(dmts_state *stt) {
    StateInternal *si = (StateInternal *)stt->internal;
    const dmts_system *sys = &stt->sys;
    SysView v;
    v.n = sys->n_atoms;
    v.n_rep = sys->n_replicas;
    v.rep_off = sys->rep_off;
    v.box = sys->box;
    v.x = sys->x;
    v.species = sys->species;
    v.mol_id = sys->mol_id;
    v.bond_ptr = sys->bond_ptr;
    v.bond_idx = sys->bond_idx;
    v.bond_r0 = sys->bond_r0;
    v.atom_rep = (int *)si->atom_rep.p;
    v.order = (const int *)si->scratch.cell_atoms.p;   // atoms sorted by cell at the last rebuild
    v.ms_part_off = (const int *)si->ms_part.p;
    return v;
}

// Rebuild of both lists, gated on si->gate (cells, full list, NC sub-list),
// then the gate is cleared.
void rebuild_lists(dmts_ctx *ctx, StateInternal *si, const SysView &v, cudaStream_t st) {
    NbrWork nw;
    prepare_nbr_work_async(ctx, si, v, nw);
    { ProfScope ps(ctx, "nbr_cells", st); nbr_cells(nw, si->r_cons, st); }
    {
        // the full list and, in the same pass, the NC list within r_nc + skin
        ProfScope ps(ctx, "nbr_fill", st);
        if (ctx->has_nc)
            nbr_fill(nw, si->r_cons, (int *)si->cons_row.p, (int *)si->cons_col.p, si->cons_cap, (float *)si->x_ref.p,
                     st, si->r_nc, (int *)si->nc_row.p, (int *)si->nc_col.p, si->nc_cap);
        else
            nbr_fill(nw, si->r_cons, (int *)si->cons_row.p, (int *)si->cons_col.p, si->cons_cap, (float *)si->x_ref.p,
                     st);
    }
    k_set_int<<<1, 1, 0, st>>>((int *)si->gate.p, 0);
    count_launch();
}

void prepare_nbr_work_async(dmts_ctx *ctx, StateInternal *si, const SysView &v, NbrWork &nw) {
    NbrScratch &b = si->scratch;
    nw.n_atoms = v.n;
    nw.n_rep = v.n_rep;
    nw.n_cells = si->n_cells;
    nw.x = v.x;
    nw.rep_off = v.rep_off;
    nw.atom_rep = v.atom_rep;
    nw.grid = (CellGrid *)b.grid.p;
    nw.cell_cnt = (int *)b.cell_cnt.p;
    nw.cell_start = (int *)b.cell_start.p;
    nw.cell_atoms = (int *)b.cell_atoms.p;
    nw.atom_cell = (int *)b.atom_cell.p;
    nw.atom_slot = (int *)b.atom_slot.p;
    nw.counts = (int *)b.counts.p;
    nw.counts_sub = (int *)b.counts_sub.p;
    nw.slots = b.slots.p ? (int *)b.slots.p : nullptr;
    nw.slot_cap = kNbrSlots;
    nw.total = (long long *)b.total.p;
    nw.gate = (int *)si->gate.p;
    nw.err = ctx->d_err;
    nw.box = v.box;
    // sized when the state was set up (prepare_nbr_work)
    nw.scan_status = (unsigned long long *)b.scan.p;
    nw.scan_counter = nw.scan_status + 2 * (size_t)b.scan_tiles;
    nw.scan_tiles = b.scan_tiles;
}

}  // namespace dmts

// Stream-ordered host copies of the replica offsets and boxes.
static bool host_copy_offsets(dmts_ctx *ctx, const dmts_system *sys, std::vector<int> &rep_off,
                              std::vector<float> &box, cudaStream_t st) {
    rep_off.resize(sys->n_replicas + 1);
    box.resize(3 * sys->n_replicas);
    return ck(ctx, cudaMemcpyAsync(rep_off.data(), sys->rep_off, sizeof(int) * rep_off.size(), cudaMemcpyDeviceToHost, st),
              "rep_off copy") &&
           ck(ctx, cudaMemcpyAsync(box.data(), sys->box, sizeof(float) * box.size(), cudaMemcpyDeviceToHost, st),
              "box copy") &&
           ck(ctx, cudaStreamSynchronize(st), "offsets");
}

// Prefix-scan scratch for scans of up to n elements (status words and tile
// counters, zero on allocation) and its fields of `nw`.
static bool scan_scratch(dmts_ctx *ctx, NbrScratch &b, int n, NbrWork &nw, cudaStream_t st) {
    const int tiles = scan_tiles_for(n);
    if (tiles > b.scan_tiles) {
        b.scan.release();
        const size_t bytes = sizeof(unsigned long long) * (2 * (size_t)tiles + 2);
        if (!b.scan.ensure(bytes) || !ck(ctx, cudaMemsetAsync(b.scan.p, 0, bytes, st), "scan scratch")) return false;
        b.scan_tiles = tiles;
    }
    nw.scan_status = (unsigned long long *)b.scan.p;
    nw.scan_counter = nw.scan_status + 2 * (size_t)b.scan_tiles;
    nw.scan_tiles = b.scan_tiles;
    return true;
}

// Builds the cell structure for `grids` into `nw` scratch owned by `bufs`.
static dmts_status prepare_nbr_work(dmts_ctx *ctx, NbrScratch &b, const SysView &v, const std::vector<CellGrid> &grids,
                                    int n_cells, const int *gate, NbrWork &nw, cudaStream_t st) {
    const int N = v.n, R = v.n_rep;
    if (!b.grid.ensure(sizeof(CellGrid) * R) || !b.cell_cnt.ensure(sizeof(int) * (n_cells + 1)) ||
        !b.cell_start.ensure(sizeof(int) * (n_cells + 1)) || !b.cell_atoms.ensure(sizeof(int) * (N + 1)) ||
        !b.atom_cell.ensure(sizeof(int) * (N + 1)) || !b.atom_slot.ensure(sizeof(int) * (N + 1)) ||
        !b.counts.ensure(sizeof(int) * (N + 1)) || !b.counts_sub.ensure(sizeof(int) * (N + 1)) ||
        !b.total.ensure(sizeof(long long)))
        return fail(ctx, DMTS_E_OOM, "neighbour scratch allocation failed");
    if (!ck(ctx, cudaMemcpyAsync(b.grid.p, grids.data(), sizeof(CellGrid) * R, cudaMemcpyHostToDevice, st), "grid upload") ||
        !ck(ctx, cudaStreamSynchronize(st), "grid upload"))
        return DMTS_E_CUDA;
    nw.n_atoms = N;
    nw.n_rep = R;
    nw.n_cells = n_cells;
    nw.x = v.x;
    nw.rep_off = v.rep_off;
    nw.atom_rep = v.atom_rep;
    nw.grid = (CellGrid *)b.grid.p;
    nw.cell_cnt = (int *)b.cell_cnt.p;
    nw.cell_start = (int *)b.cell_start.p;
    nw.cell_atoms = (int *)b.cell_atoms.p;
    nw.atom_cell = (int *)b.atom_cell.p;
    nw.atom_slot = (int *)b.atom_slot.p;
    nw.counts = (int *)b.counts.p;
    nw.counts_sub = (int *)b.counts_sub.p;
    nw.total = (long long *)b.total.p;
    nw.gate = gate;
    nw.err = ctx->d_err;
    if (!scan_scratch(ctx, b, std::max(N, n_cells), nw, st)) return fail(ctx, DMTS_E_OOM, "scan scratch allocation failed");
    return DMTS_OK;
}

void free_state_internal(StateInternal *si) {
    if (!si) return;
    if (si->call_graph) cudaGraphExecDestroy(si->call_graph);
    si->cons_row.release();
    si->cons_col.release();
    si->nc_row.release();
    si->nc_col.release();
    si->x_ref.release();
    si->gate.release();
    si->atom_rep.release();
    si->ms_part.release();
    si->baro_ke.release();
    si->thermo_part.release();
    si->baro_K.release();
    si->baro_f.release();
    si->scratch.release_all();
    delete si;
}

// Allocates lists (capacity from a first count with 40 % head-room) and the
// cell grids; leaves the lists built for the current positions.
dmts_status init_state(dmts_ctx *ctx, dmts_state *stt, float skin, cudaStream_t st, float grid_margin) {
    const dmts_system *sys = &stt->sys;
    StateInternal *si = (StateInternal *)stt->internal;
    if (!si) {
        si = new StateInternal();
        stt->internal = si;
    }
    std::vector<int> rep_off;
    std::vector<float> box;
    if (!host_copy_offsets(ctx, sys, rep_off, box, st)) return DMTS_E_CUDA;
    if (rep_off[0] != 0 || rep_off.back() != sys->n_atoms) return fail(ctx, DMTS_E_INVALID, "rep_off inconsistent");
    si->n = sys->n_atoms;
    si->n_rep = sys->n_replicas;
    si->skin = skin;
    si->grid_margin = grid_margin;
    si->r_cons = std::max(ctx->cons.rc, ctx->prior.lj_rc) + skin;
    si->r_nc = (ctx->has_nc ? ctx->nc.rc : 0.f) + skin;
    dmts_status s = setup_grids(ctx, rep_off, box, si->r_cons, si->grids, si->n_cells, grid_margin);
    if (s != DMTS_OK) return s;
    const int N = si->n;
    if (!si->atom_rep.ensure(sizeof(int) * (N + 1)) || !si->x_ref.ensure(sizeof(float) * 3 * (N + 1)) ||
        !si->gate.ensure(sizeof(int)) || !si->cons_row.ensure(sizeof(int) * (N + 1)) ||
        !si->nc_row.ensure(sizeof(int) * (N + 1)) || !si->ms_part.ensure(sizeof(int) * (sys->n_replicas + 1)))
        return fail(ctx, DMTS_E_OOM, "state allocation failed");
    atom_rep_map(sys->rep_off, sys->n_replicas, N, (int *)si->atom_rep.p, st);
    launch_mean_part_off(sys->rep_off, sys->n_replicas, (int *)si->ms_part.p, st);
    k_set_int<<<1, 1, 0, st>>>((int *)si->gate.p, 1);
    count_launch();
    SysView v = state_view(stt);
    NbrWork nw;
    s = prepare_nbr_work(ctx, si->scratch, v, si->grids, si->n_cells, (int *)si->gate.p, nw, st);
    if (s != DMTS_OK) return s;
    nw.box = v.box;
    nbr_cells(nw, si->r_cons, st);
    // size the lists from a count pass
    nbr_fill(nw, si->r_cons, (int *)si->cons_row.p, nullptr, -1, nullptr, st);
    long long tot = 0;
    cudaMemcpyAsync(&tot, nw.total, sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (!ck(ctx, cudaStreamSynchronize(st), "list sizing")) return DMTS_E_CUDA;
    const long long want_cons = (long long)(tot * 1.4) + 16LL * N + 1024;
    const double frac = ctx->has_nc ? std::pow(si->r_nc / si->r_cons, 3.0) : 0.0;
    const long long want_nc = (long long)(tot * frac * 1.6) + 16LL * N + 1024;
    if (!si->cons_col.ensure(sizeof(int) * want_cons) || !si->nc_col.ensure(sizeof(int) * want_nc) ||
        !si->scratch.slots.ensure(sizeof(int) * (size_t)N * kNbrSlots))
        return fail(ctx, DMTS_E_OOM, "neighbour list allocation failed");
    si->cons_cap = (long long)(si->cons_col.cap / sizeof(int));
    si->nc_cap = (long long)(si->nc_col.cap / sizeof(int));
    rebuild_lists(ctx, si, v, st);
    int err = 0;
    cudaMemcpyAsync(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!ck(ctx, cudaStreamSynchronize(st), "initial lists")) return DMTS_E_CUDA;
    if (err) return fail(ctx, (dmts_status)err, "initial neighbour build failed");
    return DMTS_OK;
}


// ================================================================ C ABI ==
extern "C" {

dmts_status dmts_create(dmts_ctx **out, const dmts_model *cons, const dmts_model *nc, const dmts_prior *prior,
                        int device) {
    if (!out) return fail(nullptr, DMTS_E_INVALID, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(nullptr, DMTS_E_CUDA, "no such CUDA device");
    if (cudaSetDevice(device) != cudaSuccess) return fail(nullptr, DMTS_E_CUDA, "cudaSetDevice failed");
    dmts_ctx *ctx = new dmts_ctx();
    ctx->device = device;
    if (prior) ctx->prior = *prior;
    else ctx->prior = {450.f, 0.15f, 3.15f, 5.f, 6.f, 3.5f, 6.f};
    if (ctx->prior.rep_rc > 0.f && (ctx->prior.rep_p < 2.f || ctx->prior.rep_p > 12.f)) {
        delete ctx;
        return fail(nullptr, DMTS_E_INVALID, "rep_p must be in 2..12");
    }
    if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess) {
        delete ctx;
        return fail(nullptr, DMTS_E_OOM, "allocation failed");
    }
    cudaMemset(ctx->d_err, 0, sizeof(int));
    if (cons) {
        dmts_status s = load_model(ctx, cons, false, ctx->cons);
        if (s != DMTS_OK) {
            std::string msg = ctx->last_error;
            dmts_destroy(ctx);
            return fail(nullptr, s, msg);
        }
        ctx->has_cons = true;
    }
    if (nc) {
        dmts_status s = load_model(ctx, nc, true, ctx->nc);
        if (s != DMTS_OK) {
            std::string msg = ctx->last_error;
            dmts_destroy(ctx);
            return fail(nullptr, s, msg);
        }
        ctx->has_nc = true;
        if (ctx->prior.rep_rc > ctx->nc.rc) {
            dmts_destroy(ctx);
            return fail(nullptr, DMTS_E_INVALID, "rep_rc must not exceed the NC cutoff");
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        dmts_destroy(ctx);
        return fail(nullptr, DMTS_E_CUDA, "device error during set-up");
    }
    *out = ctx;
    return DMTS_OK;
}

void dmts_destroy(dmts_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->cons.dev) cudaFree(ctx->cons.dev);
    if (ctx->nc.dev) cudaFree(ctx->nc.dev);
    if (ctx->cons.dev_bf) cudaFree(ctx->cons.dev_bf);
    if (ctx->nc.dev_bf) cudaFree(ctx->nc.dev_bf);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    ctx->ws.release_all();
    ctx->nbr_scratch.release_all();
    ctx->prof.release();
    delete ctx;
}

const char *dmts_last_error(const dmts_ctx *ctx) {
    return ctx ? ctx->last_error.c_str() : g_tls_error.c_str();
}

dmts_status dmts_sync(dmts_ctx *ctx, void *stream) {
    if (!ctx) return DMTS_E_INVALID;
    cudaSetDevice(ctx->device);
    if (!ck(ctx, cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize")) return DMTS_E_CUDA;
    int err = 0;
    if (!ck(ctx, cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word")) return DMTS_E_CUDA;
    if (err) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        cudaDeviceSynchronize();
        return fail(ctx, (dmts_status)err,
                    err == DMTS_E_NBR_OVERFLOW ? "neighbour list overflow" :
                    err == DMTS_E_NONFINITE ? "non-finite positions or velocities" : "device error");
    }
    return DMTS_OK;
}

static dmts_status check_sys(dmts_ctx *ctx, const dmts_system *sys) {
    if (!ctx || !sys) return fail(ctx, DMTS_E_INVALID, "NULL argument");
    if (sys->n_atoms < 0 || sys->n_replicas < 1) return fail(ctx, DMTS_E_INVALID, "bad sizes");
    if (!sys->rep_off || !sys->box || (sys->n_atoms > 0 && (!sys->x || !sys->species || !sys->mol_id)))
        return fail(ctx, DMTS_E_INVALID, "missing system array");
    return DMTS_OK;
}

static SysView make_view(dmts_ctx *ctx, const dmts_system *sys, cudaStream_t st) {
    SysView v;
    v.n = sys->n_atoms;
    v.n_rep = sys->n_replicas;
    v.rep_off = sys->rep_off;
    v.box = sys->box;
    v.x = sys->x;
    v.species = sys->species;
    v.mol_id = sys->mol_id;
    v.bond_ptr = sys->bond_ptr;
    v.bond_idx = sys->bond_idx;
    v.bond_r0 = sys->bond_r0;
    ctx->ws.atom_rep.ensure(sizeof(int) * (v.n + 1));
    v.atom_rep = (int *)ctx->ws.atom_rep.p;
    v.order = nullptr;
    atom_rep_map(sys->rep_off, sys->n_replicas, v.n, (int *)ctx->ws.atom_rep.p, st);
    return v;
}

dmts_status nbr_build(dmts_ctx *ctx, const dmts_system *sys, dmts_nbr *nbr, long long *n_pairs, void *stream) {
    dmts_status s = check_sys(ctx, sys);
    if (s != DMTS_OK) return s;
    if (!nbr || !nbr->row_ptr || (!nbr->col && nbr->capacity > 0) || !(nbr->r_list > 0.f))
        return fail(ctx, DMTS_E_INVALID, "bad neighbour-list argument");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> rep_off;
    std::vector<float> box;
    if (!host_copy_offsets(ctx, sys, rep_off, box, st)) return DMTS_E_CUDA;
    if (rep_off[0] != 0 || rep_off.back() != sys->n_atoms) return fail(ctx, DMTS_E_INVALID, "rep_off inconsistent");
    std::vector<CellGrid> grids;
    int n_cells = 0;
    s = setup_grids(ctx, rep_off, box, nbr->r_list, grids, n_cells);
    if (s != DMTS_OK) return s;
    SysView v = make_view(ctx, sys, st);
    NbrWork nw;
    s = prepare_nbr_work(ctx, ctx->nbr_scratch, v, grids, n_cells, nullptr, nw, st);
    if (s != DMTS_OK) return s;
    if (sys->n_atoms == 0) {
        // nothing to launch: the one row offset is 0 and there are no pairs
        if (!ck(ctx, cudaMemsetAsync(nbr->row_ptr, 0, sizeof(int), st), "row_ptr") ||
            !ck(ctx, cudaStreamSynchronize(st), "nbr_build"))
            return DMTS_E_CUDA;
        if (n_pairs) *n_pairs = 0;
        return DMTS_OK;
    }
    nbr_cells(nw, nbr->r_list, st);
    nbr_fill(nw, nbr->r_list, nbr->row_ptr, nbr->col, nbr->capacity, nullptr, st);
    long long tot = 0;
    if (!ck(ctx, cudaMemcpyAsync(&tot, nw.total, sizeof(long long), cudaMemcpyDeviceToHost, st), "count copy") ||
        !ck(ctx, cudaStreamSynchronize(st), "nbr_build"))
        return DMTS_E_CUDA;
    if (n_pairs) *n_pairs = tot;
    int err = 0;
    cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        if (err == DMTS_E_NBR_OVERFLOW)
            return fail(ctx, DMTS_E_NBR_OVERFLOW, "neighbour list capacity too small");
        return fail(ctx, (dmts_status)err, "device error");
    }
    return DMTS_OK;
}

dmts_status energy_forces_cons(dmts_ctx *ctx, const dmts_system *sys, const dmts_nbr *nbr, double *energy,
                               float *forces, double *virial, int flags, void *stream) {
    dmts_status s = check_sys(ctx, sys);
    if (s != DMTS_OK) return s;
    if (!ctx->has_cons) return fail(ctx, DMTS_E_INVALID, "context has no conservative model");
    if (!nbr || !nbr->row_ptr || !nbr->col) return fail(ctx, DMTS_E_INVALID, "bad neighbour list");
    if (virial && !forces) return fail(ctx, DMTS_E_INVALID, "the virial needs the forces");
    if (nbr->r_list < ctx->cons.rc || ((flags & DMTS_WITH_PRIOR) && nbr->r_list < ctx->prior.lj_rc))
        return fail(ctx, DMTS_E_INVALID, "neighbour list cutoff below the model cutoff");
    if ((flags & DMTS_WITH_PRIOR) && sys->n_atoms > 0 && (!sys->bond_ptr || !sys->bond_idx || !sys->bond_r0))
        return fail(ctx, DMTS_E_INVALID, "prior requested without a bond table");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    SysView v = make_view(ctx, sys, st);
    s = cons_eval(ctx, v, nbr->row_ptr, nbr->col, energy, forces, flags & ~kFlagEmbedded, st, virial);
    if (s != DMTS_OK) return s;
    return ck(ctx, cudaGetLastError(), "energy_forces_cons launch") ? DMTS_OK : DMTS_E_CUDA;
}

dmts_status forces_nc(dmts_ctx *ctx, const dmts_system *sys, const dmts_nbr *nbr, float *forces, double *net_force,
                      double *virial, int flags, void *stream) {
    dmts_status s = check_sys(ctx, sys);
    if (s != DMTS_OK) return s;
    if (!ctx->has_nc) return fail(ctx, DMTS_E_INVALID, "context has no NC model");
    if (!nbr || !nbr->row_ptr || !nbr->col || !forces) return fail(ctx, DMTS_E_INVALID, "bad argument");
    if (nbr->r_list < ctx->nc.rc) return fail(ctx, DMTS_E_INVALID, "neighbour list cutoff below the NC cutoff");
    if ((flags & DMTS_WITH_BONDS) && sys->n_atoms > 0 && (!sys->bond_ptr || !sys->bond_idx || !sys->bond_r0))
        return fail(ctx, DMTS_E_INVALID, "bonds requested without a bond table");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    SysView v = make_view(ctx, sys, st);
    s = nc_eval(ctx, v, nbr->row_ptr, nbr->col, forces, net_force, flags & ~kFlagEmbedded, st, virial, 0);
    if (s != DMTS_OK) return s;
    return ck(ctx, cudaGetLastError(), "forces_nc launch") ? DMTS_OK : DMTS_E_CUDA;
}

// ------------------------------------------------------------ respa_step
void dmts_state_release(dmts_ctx *ctx, dmts_state *st) {
    if (!st || !st->internal) return;
    if (ctx) cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    free_state_internal((StateInternal *)st->internal);
    st->internal = nullptr;
}

dmts_status nc_distill_step(dmts_ctx *ctx, const dmts_system *sys, const dmts_nbr *nbr, const float *target,
                            int params, float lr, int adam_step, double *loss, float *grad, void *stream) {
    dmts_status s = check_sys(ctx, sys);
    if (s != DMTS_OK) return s;
    if (!ctx->has_nc) return fail(ctx, DMTS_E_INVALID, "context has no NC model");
    if (!nbr || !nbr->row_ptr || !nbr->col || !target) return fail(ctx, DMTS_E_INVALID, "bad argument");
    if (nbr->r_list < ctx->nc.rc) return fail(ctx, DMTS_E_INVALID, "neighbour list cutoff below the NC cutoff");
    if (params & ~(DMTS_FIT_QK | DMTS_FIT_MLP | DMTS_FIT_LAYER)) return fail(ctx, DMTS_E_INVALID, "unknown weights to fit");
    if (lr > 0.f && adam_step < 1) return fail(ctx, DMTS_E_INVALID, "adam_step counts from 1");
    if (sys->n_atoms > 0 && (!sys->bond_ptr || !sys->bond_idx || !sys->bond_r0))
        return fail(ctx, DMTS_E_INVALID, "missing bond table");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const SysView v = make_view(ctx, sys, st);
    DevModel &m = ctx->nc;
    Workspace &w = ctx->ws;
    const int N = v.n, H = m.K + m.nl, QKW = 2 * H * m.nc, C = m.C;
    const bool fit_mlp = params & DMTS_FIT_MLP, fit_qk = params & DMTS_FIT_QK, fit_layer = params & DMTS_FIT_LAYER;
    const size_t nb = m.n_weights, part = std::max((size_t)64 * QKW * (C + 1) + (size_t)64 * C * (2 * C + 1),
                                                   (size_t)1024 * 2 * m.K * C);
    if (!w.dist_F.ensure(sizeof(float) * 3 * (N + 1)) || !w.dist_g.ensure(sizeof(float) * 3 * (N + 1)) ||
        !w.dist_sq.ensure(sizeof(float) * (N + 1)) || !w.dist_gqk.ensure(sizeof(float) * ((size_t)QKW * N + 1)) ||
        !w.dist_gs1.ensure(sizeof(float) * ((size_t)C * N + 1)) || !w.dist_gh.ensure(sizeof(float) * ((size_t)C * N + 1)) ||
        !w.dist_h.ensure(sizeof(float) * ((size_t)C * N + 1)) || !w.dist_dw.ensure(sizeof(float) * nb) ||
        !w.adam_m.ensure(sizeof(float) * nb) || !w.adam_v.ensure(sizeof(float) * nb) ||
        !w.dist_part.ensure(sizeof(float) * part) || !w.ms_scratch.ensure(mean_sub_scratch_bytes(N, v.n_rep)) ||
        !w.dist_A.ensure(sizeof(float) * ((size_t)4 * C * N + 1)) || !w.dist_gq.ensure(sizeof(float) * ((size_t)2 * C * N + 1)) ||
        !w.dist_gv.ensure(sizeof(float) * ((size_t)3 * m.nl * N + 1)))
        return fail(ctx, DMTS_E_OOM, "workspace allocation failed");
    // forward: the fast force (it leaves q, the MLP's activations and
    // pre-activations, the layer features, the q/k rows and V in the workspace)
    s = nc_eval(ctx, v, nbr->row_ptr, nbr->col, (float *)w.dist_F.p, nullptr, DMTS_WITH_BONDS | kFlagKeepPre, st);
    if (s != DMTS_OK) return s;
    launch_distill_residual(N, (const float *)w.dist_F.p, target, (float *)w.dist_g.p, (float *)w.dist_sq.p, st);
    if (loss) launch_replica_sum((const float *)w.dist_sq.p, v.rep_off, v.n_rep, loss, 0, st);
    // adjoint of the mean subtraction: the gradient minus its replica mean
    launch_mean_sub((float *)w.dist_g.p, (float *)w.dist_g.p, v.rep_off, v.n_rep, N, nullptr, w.ms_scratch.p, ctx->d_err,
                    st);
    NCHeadArgs a;
    memset(&a, 0, sizeof a);
    a.x = v.x;
    a.atom_rep = v.atom_rep;
    a.box = v.box;
    a.row_ptr = nbr->row_ptr;
    a.col = nbr->col;
    a.n_atoms = N;
    a.rc = m.rc;
    a.inv_rc = 1.f / m.rc;
    a.bnorm = sqrtf(2.f / m.rc);
    a.p = m.p;
    a.QK = (const float *)w.nc_qk.p;
    a.V = (const float *)w.nc_v.p;
    a.scale = m.scale;
    a.order = v.order;
    a.err = ctx->d_err;
    float *gqk = (float *)w.dist_gqk.p, *gs1 = (float *)w.dist_gs1.p, *gh = (float *)w.dist_gh.p;
    launch_nc_head_bwd(m.K, m.nc, m.nl, a, (const float *)w.dist_g.p, gqk, fit_layer ? (float *)w.dist_gv.p : nullptr,
                       st);
    // weight gradients in the blob's layout (zero where not fitted)
    float *dw = grad ? grad : (float *)w.dist_dw.p;
    if (!ck(ctx, cudaMemsetAsync(dw, 0, sizeof(float) * nb, st), "gradient reset")) return DMTS_E_CUDA;
    auto at = [&](const float *p) { return dw + (p - m.dev); };
    const float *s1 = (const float *)w.nc_s.p + (size_t)N * C;
    float *part_buf = (float *)w.dist_part.p;
    if (fit_qk) launch_atb(N, QKW, C, gqk, s1, at(m.Wqk), nullptr, part_buf, st);   // dW_qk = gQK^T s1
    if (fit_mlp || fit_layer) {
        // s1 = s0 + act W2^T + b2, act = silu(h), h = q W1^T + b1
        Epi e = epi(EPI_STORE);
        e.out = gs1;
        launch_gemm_f32(N, C, QKW, gqk, m.Wqk, 0, e, st);                               // g_s1 = gQK W_qk
        Epi ed = epi(EPI_DSILU);
        ed.H = (float *)w.dist_h.p;
        ed.out = gh;
        launch_gemm_f32(N, C, C, gs1, m.w2[0], 0, ed, st);                             // g_h = (g_s1 W2) silu'(h)
        if (fit_mlp) {
            launch_atb(N, C, C, gs1, (const float *)w.nc_act.p, at(m.w2[0]), at(m.b2[0]), part_buf, st);
            launch_atb(N, C, 2 * C, gh, (const float *)w.nc_q.p, at(m.w1[0]), at(m.b1[0]), part_buf, st);
        }
    }
    if (fit_layer) {
        // q = (A_00^2, sum_m A_1m^2) per channel, V_t = sum_c U[t][c] A_1m[c]
        Epi e = epi(EPI_STORE);
        e.out = (float *)w.dist_gq.p;
        launch_gemm_f32(N, 2 * C, C, gh, m.w1[0], 0, e, st);                           // g_q = g_h W1
        launch_nc_dU(N, C, m.nl, (const float *)w.dist_gv.p, (const float *)w.dist_A.p, part_buf, at(m.U), st);
        NCLayerGradArgs la;
        la.x = v.x;
        la.atom_rep = v.atom_rep;
        la.box = v.box;
        la.row_ptr = nbr->row_ptr;
        la.col = nbr->col;
        la.n_atoms = N;
        la.rc = m.rc;
        la.inv_rc = 1.f / m.rc;
        la.bnorm = sqrtf(2.f / m.rc);
        la.nu = m.nu;
        la.p = m.p;
        la.s0 = (const float *)w.nc_s.p;
        la.A = (const float *)w.dist_A.p;
        la.gq = (const float *)w.dist_gq.p;
        la.gV = (const float *)w.dist_gv.p;
        la.U = m.U;
        la.n_l = m.nl;
        la.err = ctx->d_err;
        launch_nc_layer_wgrad(C, la, part_buf, at(m.wrad[0]), st);
    }
    if (lr > 0.f && params) {
        if (adam_step == 1 && (!ck(ctx, cudaMemsetAsync(w.adam_m.p, 0, sizeof(float) * nb, st), "adam reset") ||
                               !ck(ctx, cudaMemsetAsync(w.adam_v.p, 0, sizeof(float) * nb, st), "adam reset")))
            return DMTS_E_CUDA;
        // bf: the weight's split-bf16 copy (K-major, logical row length kd), refreshed after the step
        auto adam = [&](float *p, size_t n, __nv_bfloat16 *bf, int kd) {
            const size_t o = (size_t)(p - m.dev);
            launch_adam((int)n, p, dw + o, (float *)w.adam_m.p + o, (float *)w.adam_v.p + o, lr, adam_step, bf, kd,
                        st);
        };
        if (fit_qk) adam(m.Wqk, (size_t)QKW * C, m.bf16 ? m.wqk_bf : nullptr, C);
        if (fit_layer) {
            adam(m.wrad[0], (size_t)2 * m.K * C, nullptr, 1);
            adam(m.U, (size_t)m.nl * C, nullptr, 1);
        }
        if (fit_mlp) {
            adam(m.w1[0], (size_t)C * 2 * C, m.bf16 ? m.w1_bf[0] : nullptr, 2 * C);
            adam(m.b1[0], C, nullptr, 1);
            adam(m.w2[0], (size_t)C * C, m.bf16 ? m.w2_bf[0] : nullptr, C);
            adam(m.b2[0], C, nullptr, 1);
        }
    }
    return ck(ctx, cudaGetLastError(), "nc_distill_step launch") ? DMTS_OK : DMTS_E_CUDA;
}

dmts_status dmts_state_lists(dmts_ctx *ctx, const dmts_state *st, int which, int32_t *row_ptr, int32_t *col,
                             int64_t col_capacity, int64_t *n_pairs, float *r_list, void *stream) {
    if (!ctx || !st || !row_ptr || !n_pairs || (which != 0 && which != 1))
        return fail(ctx, DMTS_E_INVALID, "bad arguments");
    const StateInternal *si = (const StateInternal *)st->internal;
    if (!si) return fail(ctx, DMTS_E_INVALID, "the state holds no lists before its first respa_step");
    const Buf &rb = which == 0 ? si->cons_row : si->nc_row;
    const Buf &cb = which == 0 ? si->cons_col : si->nc_col;
    if (!rb.p) return fail(ctx, DMTS_E_INVALID, "the state holds no such list");
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = si->n;
    int total = 0;
    if (!ck(ctx, cudaMemcpyAsync(row_ptr, rb.p, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, s), "list copy") ||
        !ck(ctx, cudaMemcpyAsync(&total, (const int *)rb.p + n, sizeof(int), cudaMemcpyDeviceToHost, s), "list size") ||
        !ck(ctx, cudaStreamSynchronize(s), "list copy"))
        return DMTS_E_CUDA;
    *n_pairs = total;
    if (r_list) *r_list = which == 0 ? si->r_cons : si->r_nc;
    if (total > col_capacity) return fail(ctx, DMTS_E_NBR_OVERFLOW, "col_capacity too small");
    if (total > 0 && (!col || !ck(ctx, cudaMemcpyAsync(col, cb.p, sizeof(int) * (size_t)total, cudaMemcpyDeviceToDevice, s),
                                  "list copy")))
        return col ? DMTS_E_CUDA : fail(ctx, DMTS_E_INVALID, "col is NULL");
    return ck(ctx, cudaStreamSynchronize(s), "list copy") ? DMTS_OK : DMTS_E_CUDA;
}

static void gamma_consts(const dmts_integrator *p, double dt, float *c1, float *c2) {
    for (int s = 0; s < DMTS_MAX_SPECIES; ++s) {
        const double e = std::exp(-p->gamma_ps[s] * 1e-3 * dt);
        c1[s] = (float)e;
        c2[s] = (float)std::sqrt((1.0 - e * e) * kBoltzmann * p->temperature * kAccConvD);
    }
}

dmts_status respa_step(dmts_ctx *ctx, dmts_state *stt, const dmts_integrator *p, int n_outer, void *stream) {
    return dmts::respa_run(ctx, stt, p, n_outer, (cudaStream_t)stream, nullptr, true);
}

}  // extern "C"

// Algorithm 1 (or STS) for n_outer outer steps; fl_max (nullable, device,
// one per replica) receives the running maximum of |F - F_S| (float bits) at
// every outer kick.
// Outer steps replayed from a CUDA graph unless DMTS_CUDA_GRAPHS=0 (the
// launches are the same either way; the variable exists to compare them).
static bool graphs_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("DMTS_CUDA_GRAPHS");
        return !(e && e[0] == '0');
    }();
    return on;
}

// The context's graph stream and its two join events (created on first use).
static bool ensure_graph_stream(dmts_ctx *ctx) {
    if (ctx->gstream) return true;
    return ck(ctx, cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking), "graph stream") &&
           ck(ctx, cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming), "graph event") &&
           ck(ctx, cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming), "graph event");
}

// What a captured call depends on besides the device contents: the
// integrator's parameters, the number of outer steps, the state's arrays and
// the generation of the library's device allocations.
static std::vector<uint64_t> call_key(const dmts_integrator *p, int n_outer, const dmts_state *stt) {
    std::vector<uint64_t> k;
    auto f32 = [&](float v) { uint32_t u; memcpy(&u, &v, 4); k.push_back(u); };
    auto f64 = [&](double v) { uint64_t u; memcpy(&u, &v, 8); k.push_back(u); };
    auto ptr = [&](const void *q) { k.push_back((uint64_t)(uintptr_t)q); };
    f32(p->dt_outer);
    k.push_back((uint64_t)(uint32_t)p->n_inner);
    f32(p->temperature);
    for (int i = 0; i < DMTS_MAX_SPECIES; ++i) f64(p->gamma_ps[i]);
    k.push_back((uint64_t)(uint32_t)p->mode);
    f32(p->skin);
    k.push_back((uint64_t)(uint32_t)p->thermostat);
    k.push_back((uint64_t)(uint32_t)p->barostat);
    f32(p->pressure_atm);
    f32(p->tau_p_ps);
    k.push_back((uint64_t)(uint32_t)n_outer);
    const dmts_system &y = stt->sys;
    k.push_back((uint64_t)(uint32_t)y.n_atoms);
    k.push_back((uint64_t)(uint32_t)y.n_replicas);
    const void *arrays[] = {y.rep_off, y.box, y.x, y.species, y.mol_id, y.bond_ptr, y.bond_idx, y.bond_r0,
                            stt->v, stt->f_nc, stt->f_cons, stt->masses, stt->energy, stt->step, stt->seed,
                            stt->replica_id, stt->virial_nc, stt->virial_cons, stt->virial_est, stt->baro,
                            stt->thermo, stt->internal};
    for (const void *q : arrays) ptr(q);
    k.push_back(alloc_generation());
    return k;
}

dmts_status dmts::respa_run(dmts_ctx *ctx, dmts_state *stt, const dmts_integrator *p, int n_outer, cudaStream_t st,
                            unsigned *fl_max, bool cache_short_calls) {
    if (!stt || !p) return fail(ctx, DMTS_E_INVALID, "NULL argument");
    dmts_status s = check_sys(ctx, &stt->sys);
    if (s != DMTS_OK) return s;
    if (!ctx->has_cons) return fail(ctx, DMTS_E_INVALID, "context has no conservative model");
    const bool sts = p->mode == DMTS_MODE_STS;
    if (!sts && (!ctx->has_nc || p->n_inner < 1)) return fail(ctx, DMTS_E_INVALID, "RESPA needs an NC model and n_inner >= 1");
    if (!(p->dt_outer > 0.f) || n_outer < 0 || !(p->skin > 0.f) ||
        (p->thermostat != DMTS_LANGEVIN && p->thermostat != DMTS_FFL))
        return fail(ctx, DMTS_E_INVALID, "bad integrator parameters");
    if (!stt->v || !stt->f_cons || (!sts && !stt->f_nc) || !stt->masses || !stt->step || !stt->seed || !stt->replica_id)
        return fail(ctx, DMTS_E_INVALID, "missing state array");
    if (stt->sys.n_atoms > 0 && (!stt->sys.bond_ptr || !stt->sys.bond_idx || !stt->sys.bond_r0))
        return fail(ctx, DMTS_E_INVALID, "missing bond table");
    if (stt->virial_est && (!stt->virial_cons || (!sts && !stt->virial_nc)))
        return fail(ctx, DMTS_E_INVALID, "virial_est needs virial_cons and virial_nc");
    const bool npt = !sts && p->barostat;
    if (npt && (!stt->baro || !stt->virial_est || !(p->tau_p_ps > 0.f)))
        return fail(ctx, DMTS_E_INVALID, "the barostat needs st->baro, the virial arrays and tau_p_ps > 0");
    if ((stt->thermo || stt->thermo_trace) && !stt->energy)
        return fail(ctx, DMTS_E_INVALID, "thermo needs the energy array");
    if (stt->thermo_trace && (!stt->thermo || n_outer > stt->thermo_trace_rows))
        return fail(ctx, DMTS_E_INVALID, "thermo_trace needs thermo and at least n_outer rows");
    cudaSetDevice(ctx->device);
    if (stt->virial_est && !sts && !ctx->ws.nc_w_last.ensure(sizeof(double) * stt->sys.n_replicas))
        return fail(ctx, DMTS_E_OOM, "workspace allocation failed");
    if (!stt->internal) {
        s = init_state(ctx, stt, p->skin, st, npt ? kBaroGridMargin : 0.f);
        if (s != DMTS_OK) {
            free_state_internal((StateInternal *)stt->internal);
            stt->internal = nullptr;
            return s;
        }
    }
    StateInternal *si = (StateInternal *)stt->internal;
    if (si->n != stt->sys.n_atoms || si->n_rep != stt->sys.n_replicas || si->skin != p->skin)
        return fail(ctx, DMTS_E_INVALID, "state shape changed; release the state first");
    if (npt && si->grid_margin < kBaroGridMargin)
        return fail(ctx, DMTS_E_INVALID, "state built without the barostat's cell margin; release it first");
    if ((stt->thermo || stt->thermo_trace) &&
        !si->thermo_part.ensure(thermo_scratch_bytes(stt->sys.n_atoms, stt->sys.n_replicas)))
        return fail(ctx, DMTS_E_OOM, "thermo workspace allocation failed");
    if (npt && (!si->baro_ke.ensure(sizeof(float) * (stt->sys.n_atoms + 1)) ||
                !si->baro_K.ensure(sizeof(double) * stt->sys.n_replicas) ||
                !si->baro_f.ensure(sizeof(float) * 3 * stt->sys.n_replicas)))
        return fail(ctx, DMTS_E_OOM, "barostat workspace allocation failed");
    const SysView v = state_view(stt);
    const int *crow = (int *)si->cons_row.p, *ccol = (int *)si->cons_col.p;
    const int *nrow = (int *)si->nc_row.p, *ncol = (int *)si->nc_col.p;
    // the species embedding is computed by the first evaluation of each
    // model in this call and kept in the workspace for the others
    int cons_emb = 0, nc_emb = 0;
    auto cons_full = [&]() {
        const dmts_status r = cons_eval(ctx, v, crow, ccol, stt->energy, stt->f_cons, DMTS_WITH_PRIOR | cons_emb, st,
                                        stt->virial_cons);
        cons_emb = kFlagEmbedded;
        return r;
    };
    // fast force; inside the inner loop it also adds its virial proxy to the
    // per-replica average of the outer step (Sec. 2, virial term in NPT)
    // The fast force's mean subtraction is left to the next integrator launch
    // (or the kinetic-energy reduction before it), which reads the head's
    // force and the replica means and stores the subtracted force in
    // stt->f_nc: one launch and one pass over the forces less per inner step.
    bool mean_pending = false;
    auto nc_fast_on = [&](bool with_virial, cudaStream_t s_nc) {
        const dmts_status r = nc_eval(ctx, v, nrow, ncol, stt->f_nc, nullptr, DMTS_WITH_BONDS | nc_emb | kFlagDeferMean,
                                      s_nc, with_virial ? stt->virial_nc : nullptr, 1);
        nc_emb = kFlagEmbedded;
        mean_pending = true;
        return r;
    };
    auto nc_fast = [&](bool with_virial) { return nc_fast_on(with_virial, st); };
    // the last NC evaluation of an outer step and the conservative one are
    // both at the step's final positions and share no buffer: the first runs
    // on the context's second stream, forked after the list rebuild and
    // joined before the next integrator launch
    const bool overlap = !sts;
    if (overlap && !ctx->aux &&
        (!ck(ctx, cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking), "second stream") ||
         !ck(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming), "fork event") ||
         !ck(ctx, cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming), "join event")))
        return DMTS_E_CUDA;
    auto integrate = [&](IntegArgs a) {
        if (mean_pending) {
            a.fast_pre = (const float *)ctx->ws.nc_f.p;
            a.fast_sum = (const unsigned long long *)ctx->ws.nc_sum.p;
            a.fast_out = stt->f_nc;
            mean_pending = false;
        }
        launch_integrate(a, st);
    };

    if (stt->first_step) {
        if (!sts) {
            s = nc_fast(false);
            if (s != DMTS_OK) return s;
        }
        s = cons_full();
        if (s != DMTS_OK) return s;
        stt->first_step = 0;
    }
    IntegArgs ia;
    memset(&ia, 0, sizeof ia);
    ia.n_atoms = v.n;
    ia.atom_rep = v.atom_rep;
    ia.rep_off = v.rep_off;
    ia.x = stt->sys.x;
    ia.v = stt->v;
    ia.f_slow = stt->f_cons;
    ia.f_fast = sts ? stt->f_cons : stt->f_nc;
    ia.masses = stt->masses;
    ia.species = stt->sys.species;
    ia.seed = stt->seed;
    ia.rep_id = stt->replica_id;
    ia.step = stt->step;
    ia.x_ref = (float *)si->x_ref.p;
    ia.half_skin2 = 0.25f * p->skin * p->skin;
    ia.rebuild = (int *)si->gate.p;
    ia.err = ctx->d_err;
    ia.ffl = p->thermostat == DMTS_FFL;
    ia.fl_max = sts ? nullptr : fl_max;
    const int n_in = sts ? 1 : p->n_inner;
    const double delta = sts ? p->dt_outer : (double)p->dt_outer / n_in;
    gamma_consts(p, delta, ia.c1, ia.c2);
    ia.h_in = (float)(0.5 * delta);
    ia.h_out = 0.5f * p->dt_outer;
    if (n_outer == 0) {
        if (mean_pending) {   // first forces only: store the subtracted fast force
            IntegArgs a0 = ia;
            a0.ops = 0;
            integrate(a0);
        }
        return ck(ctx, cudaGetLastError(), "respa_step launch") ? DMTS_OK : DMTS_E_CUDA;
    }
    // A call of one or two outer steps (the loop of a caller that copies
    // the state in and out between calls) is replayed whole from a graph the
    // state keeps, captured from its first such call: the key holds the
    // integrator's parameters, the number of steps, every array of the state
    // and the generation of the library's device allocations, so a graph is
    // never replayed on arrays that moved or were freed.
    const bool cache_call = cache_short_calls && n_outer <= 2 && !ctx->prof.on && !stt->thermo_trace && !fl_max &&
                            graphs_enabled() && !ctx->graphs_off;
    if (cache_call && si->call_graph && si->call_key == call_key(p, n_outer, stt)) {
        if (!ensure_graph_stream(ctx) || !ck(ctx, cudaEventRecord(ctx->ev_in, st), "graph stream") ||
            !ck(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0), "graph stream") ||
            !ck(ctx, cudaGraphLaunch(si->call_graph, ctx->gstream), "graph launch") ||
            !ck(ctx, cudaEventRecord(ctx->ev_out, ctx->gstream), "graph stream") ||
            !ck(ctx, cudaStreamWaitEvent(st, ctx->ev_out, 0), "graph stream"))
            return DMTS_E_CUDA;
        count_launches(si->call_launches);
        return DMTS_OK;
    }
    auto rest_of_call = [&](bool step_graphs) -> dmts_status {
        // FP64 K, U + K and T per replica (pending closing kicks selected per call site)
        ThermoArgs ta;
        memset(&ta, 0, sizeof ta);
        ta.rep_off = v.rep_off;
        ta.v = stt->v;
        ta.f_fast = ia.f_fast;
        ta.f_slow = stt->f_cons;
        ta.masses = stt->masses;
        ta.h_in = ia.h_in;
        ta.h_out = ia.h_out;
        ta.energy = stt->energy;
        ta.out = stt->thermo;
        ta.part_off = v.ms_part_off;
        ta.partial = (double *)si->thermo_part.p;
        ta.n_rep = v.n_rep;
        auto thermo = [&](bool pending, double *trace_row) {
            ThermoArgs t = ta;
            t.close_b = pending;
            t.kick_l = pending && !sts;
            t.trace = trace_row;
            if (pending && mean_pending) {
                t.f_fast = (const float *)ctx->ws.nc_f.p;
                t.fast_sum = (const unsigned long long *)ctx->ws.nc_sum.p;
            }
            ProfScope ps(ctx, "thermo", st);
            launch_thermo(t, v.n, v.n_rep, st);
        };
        BaroArgs ba;
        memset(&ba, 0, sizeof ba);
        if (npt) {
            ba.n_rep = v.n_rep;
            ba.rep_off = v.rep_off;
            ba.baro = stt->baro;
            ba.box = const_cast<float *>(stt->sys.box);
            ba.K = (const double *)si->baro_K.p;
            ba.baro_f = (float *)si->baro_f.p;
            ba.seed = stt->seed;
            ba.rep_id = stt->replica_id;
            ba.step = stt->step;
            ba.delta_outer = p->dt_outer;
            ba.h = 0.5 * delta;
            ba.p_kcal = (double)p->pressure_atm * kKcalPerA3PerAtm;
            ba.tau_fs = (double)p->tau_p_ps * 1e3;
            ba.kT = kBoltzmann * p->temperature;
            ba.err = ctx->d_err;
            ia.baro_f = (const float *)si->baro_f.p;
            ia.box = ba.box;
            // kinetic energy now, for a piston force not yet set (the full force's virial)
            IntegArgs ik = ia;
            ik.ops = 0;
            ik.baro_f = nullptr;
            ik.ke = (float *)si->baro_ke.p;
            integrate(ik);
            launch_replica_sum((const float *)si->baro_ke.p, v.rep_off, v.n_rep, (double *)si->baro_K.p, 0, st);
        }
        // outer steps not timed under a sampling profiler; calls outside the loop are
        struct ActiveReset {
            dmts_ctx *c;
            ~ActiveReset() { c->prof.active = true; }
        } active_reset{ctx};
        // one outer step; its launches depend on o only through o == 0 (the
        // first inner step's kicks) and the trace row, so every later step is
        // the same sequence of launches with the same arguments
        auto outer_step = [&](int o) -> dmts_status {
            dmts_status r;
            if (!sts && stt->virial_nc &&
                !ck(ctx, cudaMemsetAsync(stt->virial_nc, 0, sizeof(double) * v.n_rep, st), "virial reset"))
                return DMTS_E_CUDA;
            if (npt) {
                ba.wvir = stt->virial_cons;
                launch_baro_start(ba, st);
            }
            for (int k = 0; k < n_in; ++k) {
                if (sts) ia.ops = (o == 0 ? 0 : OP_CLOSE_B) | OP_BAOA;
                else if (k == 0 && npt) ia.ops = OP_KICK_L2 | OP_BAOA;   // the previous step closed itself
                else if (k == 0) ia.ops = (o == 0 ? OP_KICK_L2 : (OP_CLOSE_B | OP_KICK_L | OP_KICK_L2)) | OP_BAOA;
                else ia.ops = OP_CLOSE_B | OP_BAOA;
                ia.step_add = (uint64_t)k;   // the replicas' step counters advance at the end of each outer step
                { ProfScope ps(ctx, "integrate", st); integrate(ia); }
                rebuild_lists(ctx, si, v, st);
                if (!sts) {
                    const bool last = k == n_in - 1;
                    cudaStream_t s_nc = st;
                    if (last && overlap) {
                        s_nc = ctx->aux;
                        if (!ck(ctx, cudaEventRecord(ctx->ev_fork, st), "fork") ||
                            !ck(ctx, cudaStreamWaitEvent(s_nc, ctx->ev_fork, 0), "fork"))
                            return DMTS_E_CUDA;
                    }
                    r = nc_fast_on(stt->virial_nc != nullptr, s_nc);
                    if (r != DMTS_OK) return r;
                    if (last) {
                        // the fast force's virial at the end of the outer step, for
                        // the estimator, and its average over the inner steps
                        if (stt->virial_est)
                            launch_replica_sum((const float *)ctx->ws.nc_w.p, v.rep_off, v.n_rep,
                                               (double *)ctx->ws.nc_w_last.p, 0, s_nc);
                        if (stt->virial_nc) launch_scale_d(stt->virial_nc, v.n_rep, 1.0 / n_in, s_nc);
                        if (overlap && !ck(ctx, cudaEventRecord(ctx->ev_join, s_nc), "join")) return DMTS_E_CUDA;
                    }
                }
            }
            r = cons_full();
            if (r != DMTS_OK) return r;
            if (overlap && !ck(ctx, cudaStreamWaitEvent(st, ctx->ev_join, 0), "join")) return DMTS_E_CUDA;
            if (stt->virial_est) {
                if (sts) {
                    if (!ck(ctx, cudaMemcpyAsync(stt->virial_est, stt->virial_cons, sizeof(double) * v.n_rep,
                                                 cudaMemcpyDeviceToDevice, st), "virial copy"))
                        return DMTS_E_CUDA;
                } else {
                    launch_virial_estimate(stt->virial_est, stt->virial_cons, (const double *)ctx->ws.nc_w_last.p,
                                           stt->virial_nc, v.n_rep, st);
                }
            }
            if (npt) {
                // close the outer step, then the piston's half kick with the estimator
                ia.ops = OP_CLOSE_B | OP_KICK_L;
                ia.ke = (float *)si->baro_ke.p;
                { ProfScope ps(ctx, "integrate", st); integrate(ia); }
                ia.ke = nullptr;
                launch_replica_sum((const float *)si->baro_ke.p, v.rep_off, v.n_rep, (double *)si->baro_K.p, 0, st);
                ba.wvir = stt->virial_est;
                { ProfScope ps(ctx, "barostat", st); launch_baro_end(ba, st); }
            }
            // the end of outer step o: under the barostat the step closed itself
            // above; otherwise its closing kicks are still pending
            if (stt->thermo_trace) thermo(!npt, stt->thermo_trace + (size_t)o * v.n_rep * 3);
            launch_advance_step(stt->step, v.n_rep, (uint64_t)n_in, ctx->d_err, st);
            return DMTS_OK;
        };
        // Outer steps after the first are replayed from a CUDA graph captured
        // from the second (calls of three or more steps; not with a per-step
        // trace, whose row changes, nor on the steps a sampling profiler times).
        const bool graphs = step_graphs && n_outer >= 3 && !stt->thermo_trace && graphs_enabled() && !ctx->graphs_off;
        if (graphs && !ensure_graph_stream(ctx)) return DMTS_E_CUDA;
        // the outer steps run on the context's graph stream, after everything
        // the caller's stream holds; on every way out, the caller's stream waits
        // for them and the rest of the call runs on it again
        struct StreamJoin {
            dmts_ctx *c;
            cudaStream_t *cur, user;
            bool on;
            void join() {
                if (!on) return;
                cudaEventRecord(c->ev_out, *cur);
                cudaStreamWaitEvent(user, c->ev_out, 0);
                *cur = user;
                on = false;
            }
            ~StreamJoin() { join(); }
        } sj{ctx, &st, st, false};
        cudaGraphExec_t gx = nullptr;
        unsigned long long gx_launches = 0;
        struct GraphExecReset {
            cudaGraphExec_t *g;
            ~GraphExecReset() { if (*g) cudaGraphExecDestroy(*g); }
        } gx_reset{&gx};
        if (graphs) {
            if (!ck(ctx, cudaEventRecord(ctx->ev_in, st), "graph stream") ||
                !ck(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0), "graph stream"))
                return DMTS_E_CUDA;
            st = ctx->gstream;
            sj.on = true;
        }
        bool graphs_now = graphs;
        for (int o = 0; o < n_outer; ++o) {
            if (ctx->prof.on) {
                ctx->prof.active = ctx->prof.every <= 1 || ctx->prof.outer % ctx->prof.every == 0;
                ctx->prof.outer++;
            }
            const bool replayable = graphs_now && o > 0 && !(ctx->prof.on && ctx->prof.active);
            if (replayable && gx) {
                if (!ck(ctx, cudaGraphLaunch(gx, st), "graph launch")) return DMTS_E_CUDA;
                count_launches(gx_launches);
                continue;
            }
            if (replayable) {
                // capture this step (nothing runs while capturing), then launch it
                const unsigned long long l0 = launch_count();
                if (!ck(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed), "graph capture")) return DMTS_E_CUDA;
                s = outer_step(o);
                cudaGraph_t gr = nullptr;
                const cudaError_t ce = cudaStreamEndCapture(st, &gr);
                if (s != DMTS_OK) {
                    if (gr) cudaGraphDestroy(gr);
                    return s;
                }
                const bool inst = ce == cudaSuccess && gr && cudaGraphInstantiate(&gx, gr, 0) == cudaSuccess;
                if (gr) cudaGraphDestroy(gr);
                if (!inst) {
                    // nothing ran while capturing: this context launches directly from now on
                    gx = nullptr;
                    cudaGetLastError();
                    ctx->graphs_off = true;
                    graphs_now = false;
                    s = outer_step(o);
                    if (s != DMTS_OK) return s;
                    continue;
                }
                gx_launches = launch_count() - l0;
                if (!ck(ctx, cudaGraphLaunch(gx, st), "graph launch")) return DMTS_E_CUDA;
                continue;
            }
            s = outer_step(o);
            if (s != DMTS_OK) return s;
        }
        sj.join();
        if (!npt) {
            ia.ops = sts ? OP_CLOSE_B : (OP_CLOSE_B | OP_KICK_L);
            { ProfScope ps(ctx, "integrate", st); integrate(ia); }
        }
        if (stt->thermo && !stt->thermo_trace) thermo(false, nullptr);
        return ck(ctx, cudaGetLastError(), "respa_step launch") ? DMTS_OK : DMTS_E_CUDA;
    };
    if (!cache_call) return rest_of_call(true);
    if (si->call_graph) {
        cudaGraphExecDestroy(si->call_graph);
        si->call_graph = nullptr;
    }
    // the captured call must read only the state's own arrays at entry: a
    // fast force whose mean subtraction is still pending (the first call's
    // initial forces, in the context's workspace) is stored in st->f_nc now
    if (mean_pending) {
        IntegArgs a0 = ia;
        a0.ops = 0;
        integrate(a0);
    }
    if (!ensure_graph_stream(ctx) || !ck(ctx, cudaEventRecord(ctx->ev_in, st), "graph stream") ||
        !ck(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0), "graph stream"))
        return DMTS_E_CUDA;
    const cudaStream_t user_st = st;
    st = ctx->gstream;
    // the workspace's species embedding may be another state's by the time
    // the graph is replayed: the captured call computes its own
    cons_emb = 0;
    nc_emb = 0;
    const unsigned long long l0 = launch_count();
    if (!ck(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed), "graph capture")) {
        st = user_st;
        return DMTS_E_CUDA;
    }
    s = rest_of_call(false);
    cudaGraph_t gr = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &gr);
    st = user_st;
    if (s != DMTS_OK) {
        if (gr) cudaGraphDestroy(gr);
        return s;
    }
    cudaGraphExec_t gx = nullptr;
    const bool inst = ce == cudaSuccess && gr && cudaGraphInstantiate(&gx, gr, 0) == cudaSuccess;
    if (gr) cudaGraphDestroy(gr);
    if (!inst) {
        // nothing ran while capturing: run the call directly, and launch
        // directly in this context from now on
        cudaGetLastError();
        ctx->graphs_off = true;
        return rest_of_call(false);
    }
    si->call_graph = gx;
    si->call_key = call_key(p, n_outer, stt);   // after the capture: buffers it allocated are in the key
    si->call_launches = launch_count() - l0;
    if (!ck(ctx, cudaGraphLaunch(gx, ctx->gstream), "graph launch") ||
        !ck(ctx, cudaEventRecord(ctx->ev_out, ctx->gstream), "graph stream") ||
        !ck(ctx, cudaStreamWaitEvent(st, ctx->ev_out, 0), "graph stream"))
        return DMTS_E_CUDA;
    return DMTS_OK;
}

extern "C" {

// ------------------------------------------------------------- helpers
void dmts_masses_hmr(int n, const uint8_t *species, const int *mol_id, const double *m_in, double delta_h,
                     double *m_out) {
    int max_mol = 0;
    for (int i = 0; i < n; ++i) max_mol = std::max(max_mol, mol_id[i]);
    std::vector<double> gain(max_mol + 1, 0.0), heavy(max_mol + 1, 0.0);
    for (int i = 0; i < n; ++i) {
        if (species[i] == 0) gain[mol_id[i]] += delta_h;
        else heavy[mol_id[i]] += m_in[i];
    }
    for (int i = 0; i < n; ++i) {
        const int mo = mol_id[i];
        if (heavy[mo] == 0.0) m_out[i] = m_in[i];
        else if (species[i] == 0) m_out[i] = m_in[i] + delta_h;
        else m_out[i] = m_in[i] - gain[mo] * (m_in[i] / heavy[mo]);
    }
}

dmts_status dmts_bond_table(int n_atoms, int n_bonds, const int *bonds, const float *r0, int *ptr, int *idx,
                            float *r0_out) {
    if (n_atoms < 0 || n_bonds < 0 || !ptr || (n_bonds > 0 && (!bonds || !r0 || !idx || !r0_out)))
        return DMTS_E_INVALID;
    std::vector<int> cnt(n_atoms + 1, 0);
    for (int b = 0; b < n_bonds; ++b) {
        const int i = bonds[2 * b], j = bonds[2 * b + 1];
        if (i < 0 || j < 0 || i >= n_atoms || j >= n_atoms || i == j) return DMTS_E_INVALID;
        cnt[i]++;
        cnt[j]++;
    }
    ptr[0] = 0;
    for (int i = 0; i < n_atoms; ++i) ptr[i + 1] = ptr[i] + cnt[i];
    std::vector<int> fill(ptr, ptr + n_atoms);
    for (int b = 0; b < n_bonds; ++b) {
        const int i = bonds[2 * b], j = bonds[2 * b + 1];
        idx[fill[i]] = j;
        r0_out[fill[i]++] = r0[b];
        idx[fill[j]] = i;
        r0_out[fill[j]++] = r0[b];
    }
    return DMTS_OK;
}

dmts_status dmts_contract_bf16(dmts_ctx *ctx, int M, int N, int K, const void *act, const void *wt, float *out,
                               int split, void *stream) {
    if (!ctx || !act || !wt || !out || M < 1 || !gemm_tc_supported(N, K) || (split != 0 && split != 1))
        return fail(ctx, DMTS_E_INVALID, "dmts_contract_bf16: needs M >= 1, K % 64 == 0, N % 16 == 0, split 0 or 1");
    cudaSetDevice(ctx->device);
    Epi e;
    memset(&e, 0, sizeof e);
    e.mode = EPI_STORE;
    e.out = out;
    const int r = launch_gemm_tc(M, N, K, (const __nv_bfloat16 *)act, (const __nv_bfloat16 *)wt, e, ctx->d_err,
                                 (cudaStream_t)stream, split, split ? 3 : 1);
    if (r != 0) return fail(ctx, DMTS_E_INVALID, "dmts_contract_bf16: unaligned operand or tensor map failure");
    return ck(ctx, cudaGetLastError(), "dmts_contract_bf16 launch") ? DMTS_OK : DMTS_E_CUDA;
}

// A wait that runs out: nothing arrives on this block's mbarrier.
__global__ void k_bounded_wait(uint64_t limit_ns, int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0, limit_ns)) set_error(err, DMTS_E_TIMEOUT);
}

dmts_status dmts_check_bounded_wait(dmts_ctx *ctx, int limit_us, void *stream) {
    if (!ctx || limit_us < 1 || limit_us > 1000000)
        return fail(ctx, DMTS_E_INVALID, "dmts_check_bounded_wait: limit_us must be in [1, 1000000]");
    cudaSetDevice(ctx->device);
    k_bounded_wait<<<1, 32, 0, (cudaStream_t)stream>>>((uint64_t)limit_us * 1000ull, ctx->d_err);
    count_launch();
    return ck(ctx, cudaGetLastError(), "dmts_check_bounded_wait launch") ? DMTS_OK : DMTS_E_CUDA;
}

__global__ void k_philox_words(uint64_t seed, uint32_t rep, uint64_t step, uint32_t atom0, int count, uint32_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint4 w = philox4x32_10(make_uint4(atom0 + i, rep, (uint32_t)step, (uint32_t)(step >> 32)),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    out[4 * i] = w.x; out[4 * i + 1] = w.y; out[4 * i + 2] = w.z; out[4 * i + 3] = w.w;
}

__global__ void k_gaussians(uint64_t seed, uint32_t rep, uint64_t step, uint32_t atom0, int count, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float3 g = gauss3(seed, rep, step, atom0 + i);
    out[3 * i] = g.x; out[3 * i + 1] = g.y; out[3 * i + 2] = g.z;
}

dmts_status dmts_philox_words(dmts_ctx *ctx, uint64_t seed, uint32_t replica, uint64_t step, uint32_t atom0, int count,
                              uint32_t *out, void *stream) {
    if (!ctx || !out || count < 0) return fail(ctx, DMTS_E_INVALID, "bad argument");
    cudaSetDevice(ctx->device);
    if (count) {
        k_philox_words<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(seed, replica, step, atom0, count, out);
        count_launch();
    }
    return ck(ctx, cudaGetLastError(), "philox launch") ? DMTS_OK : DMTS_E_CUDA;
}

dmts_status dmts_gaussians(dmts_ctx *ctx, uint64_t seed, uint32_t replica, uint64_t step, uint32_t atom0, int count,
                           float *out, void *stream) {
    if (!ctx || !out || count < 0) return fail(ctx, DMTS_E_INVALID, "bad argument");
    cudaSetDevice(ctx->device);
    if (count) {
        k_gaussians<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(seed, replica, step, atom0, count, out);
        count_launch();
    }
    return ck(ctx, cudaGetLastError(), "gaussian launch") ? DMTS_OK : DMTS_E_CUDA;
}

}  // extern "C"
