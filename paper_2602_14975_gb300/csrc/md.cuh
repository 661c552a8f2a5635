// NC direct-force head, analytic prior, fused BAOAB/RESPA integrator, mean
// subtraction, NPT piston and virial estimator, distillation gradients.
#pragma once
#include "common.cuh"

namespace dmts {

struct BondTable {
    const int *ptr, *idx;
    const float *r0;
    float k;
};

// Screened nuclear repulsion for species pairs (ZBL universal screening):
// E = zz[si][sj] / r * phi(r * inv_a[si][sj]) * f(r/rc; p), bonded pairs excluded.
struct RepTable {
    float zz[5][5];      // k_e Z_i Z_j
    float inv_a[5][5];   // 1 / a_ij
    float rc, inv_rc;
    int p;
    int on;
};

struct NCHeadArgs {
    const float *x;
    const int *atom_rep;
    const float *box;
    const int *row_ptr, *col;      // NC list (cutoff + skin)
    int n_atoms;
    float rc, inv_rc, bnorm;
    int p;
    const float *QK;               // [N][2][H][nc]
    const float *V;                // [N][nc_v_stride(n_l)]: the n_l 3-vectors of each atom, padded
    float scale;
    BondTable bonds;               // bonds.ptr null: no bond force, no F_rep
    RepTable rep;
    const uint8_t *species;
    unsigned long long *Ffix;      // [N][3] forces before mean subtraction, 32.32 fixed point, added to
                                   // (zero on entry; launch_nc_convert converts and clears them)
    unsigned long long *sum;       // [R][3] per-replica exact sums, cleared by the head for launch_nc_convert
    unsigned *next;                // the head's work counter (atoms taken; zero on entry, cleared by launch_nc_convert)
    int n_rep;
    float *W;                      // nullable [N]: per-atom virial proxy (pair form; each NC pair on its
                                   // lower-index atom)
    const int *order;              // nullable processing order
    int *err;                      // sticky device error word (read, and set on a timeout)
};

void launch_nc_head(int K, int n_c, int n_l, const NCHeadArgs &a, cudaStream_t st);

// Adjoint of the NC head with respect to its q/k rows (distillation): with
// gF[i] = dL/dF_i (after the mean subtraction's adjoint) writes
// gQK[i][c] = dL/dQK[i][c] ([N][2 H n_c]) and, when gV is set,
// gV[i][t][m] = dL/dV[i][t][m] ([N][n_l][3]). Uses a.x, box, lists, rc,
// bnorm, p, QK, V, scale, order, err of the forward's arguments.
void launch_nc_head_bwd(int K, int n_c, int n_l, const NCHeadArgs &a, const float *gF, float *gQK, float *gV,
                        cudaStream_t st);
// Gradients of the NC layer's weights (distillation), l_max = 1, K = 8.
struct NCLayerGradArgs {
    const float *x;
    const int *atom_rep;
    const float *box;
    const int *row_ptr, *col;      // NC list
    int n_atoms;
    float rc, inv_rc, bnorm, nu;
    int p;
    const float *s0;               // [N][C] layer input features
    const float *A;                // [N][4][C] layer output A = nu sum_j R Y s_j
    const float *gq;               // [N][2][C] dL/dq (q_l = sum_m A_lm^2)
    const float *gV;               // [N][n_l][3] dL/dV (V_t = sum_c U[t][c] A_1m[c])
    const float *U;                // [n_l][C]
    int n_l;
    const int *err;
};
// dW_rad[l][k][c] = nu sum_i sum_j gA_i[lm][c] s_j[c] Y_lm f_c B_k (lm in l), with
// gA_i = 2 A_i gq_i + (l = 1) sum_t U[t] gV_i[t][m]; part: >= 2 K C floats per
// block of the launch (at most 1,024 blocks).
void launch_nc_layer_wgrad(int C, const NCLayerGradArgs &a, float *part, float *out, cudaStream_t st);
// dU[t][c] = sum_i sum_m gV_i[t][m] A_i[1+m][c]; part: n_l C floats per slice (<= 64).
void launch_nc_dU(int n, int C, int n_l, const float *gV, const float *A, float *part, float *out, cudaStream_t st);
// Weight gradient out[o][i] = sum_a G[a][o] X[a][i] (G [N][O], X [N][I]) and,
// when cs is set, cs[o] = sum_a G[a][o]; atoms are split into slices whose
// partial sums (part: O (I + 1) floats per slice, slices <= 64) are added in
// a fixed order, so the result is deterministic.
void launch_atb(int N, int O, int I, const float *G, const float *X, float *out, float *cs, float *part,
                cudaStream_t st);
// g = 2 (F - T), sq = |F - T|^2 per atom.
void launch_distill_residual(int n, const float *F, const float *T, float *g, float *sq, cudaStream_t st);
// Adam on n parameters (fp32, moments m, v), then the split-bf16 copy
// (nullable; K-major with logical row length kd).
void launch_adam(int n, float *w, const float *grad, float *m, float *v, float lr, int step, __nv_bfloat16 *w_bf,
                 int kd, cudaStream_t st);
// v[i] *= f, i < n.
void launch_scale_d(double *v, int n, double f, cudaStream_t st);
// est[r] = cons[r] - last[r] + avg[r]
void launch_virial_estimate(double *est, const double *cons, const double *last, const double *avg, int n,
                            cudaStream_t st);
// F_out = F_in - (sum_{replica} F_in)/n_r, FP64 sums; net (nullable) [R][3].
// scratch: device memory of mean_sub_scratch_bytes(n_atoms, n_rep) bytes.
size_t mean_sub_scratch_bytes(int n_atoms, int n_rep);
// part_off (nullable): the replicas' part offsets from launch_mean_part_off,
// computed once for a fixed batch; then net must be NULL.
void launch_mean_sub(const float *F_in, float *F_out, const int *rep_off, int n_rep, int n_atoms, double *net,
                     void *scratch, const int *err, cudaStream_t st, const int *part_off = nullptr);
// part_off: device int [n_rep + 1]
void launch_mean_part_off(const int *rep_off, int n_rep, int *part_off, cudaStream_t st);
// The NC head's fixed-point forces -> fp32 F, cleared; sum[r] += the
// replica's exact integer force sum (sum cleared by the head beforehand).
void launch_nc_convert(int n, const int *atom_rep, unsigned long long *Ffix, float *F, unsigned long long *sum,
                       unsigned *next, cudaStream_t st);
// F_out = F - mean (replica means from the exact sums: sum / 2^32 / n_r in
// FP64); net (nullable) [R][3] = the sums in FP64.
void launch_nc_apply(int n, const int *atom_rep, const int *rep_off, int n_rep, const float *F, float *F_out,
                     const unsigned long long *sum, double *net, const int *err, cudaStream_t st);

struct PriorArgs {
    const float *x;
    const int *atom_rep;
    const float *box;
    const int *row_ptr, *col;      // list with cutoff >= lj_rc
    const uint8_t *species;
    const int *mol_id;
    int n_atoms;
    float lj_eps, lj_sigma, lj_rc;
    int lj_p;
    BondTable bonds;
    RepTable rep;
    float *F;                      // accumulated
    float *e_atom;                 // accumulated per-atom energy (nullable)
    float *W;                      // accumulated per-atom virial proxy, pair form (nullable)
    const int *order;              // nullable processing order
    const int *err;
};
void launch_prior(const PriorArgs &a, cudaStream_t st);

enum IntegOps {
    OP_CLOSE_B = 1,     // v += h_in a F_fast
    OP_KICK_L = 2,      // v += h_out a (F_slow - F_fast)  (end of an outer step)
    OP_KICK_L2 = 4,     // v += h_out a (F_slow - F_fast)  (start of an outer step)
    OP_BAOA = 8,        // v += h_in a F_fast; x += h_in v; O(delta); x += h_in v
};

struct IntegArgs {
    int n_atoms;
    const int *atom_rep, *rep_off;
    float *x, *v;
    const float *f_slow, *f_fast;
    const float *masses;
    const uint8_t *species;
    float c1[DMTS_MAX_SPECIES], c2[DMTS_MAX_SPECIES];
    const uint64_t *seed;
    const uint32_t *rep_id;
    const uint64_t *step;
    uint64_t step_add;
    float h_out, h_in;
    int ops;
    const float *x_ref;            // nullable: displacement check
    float half_skin2;
    int *rebuild;
    int *err;
    int ffl;                       // O-step: 0 Langevin, 1 Fast Forward Langevin
    unsigned *fl_max;              // nullable: per-replica running max of |F_slow - F_fast| (float bits)
    const float *baro_f;           // nullable: per replica [3] = e^(b h), h (e^(b h) - 1)/(b h), e^(-a h)
    float *box;                    // with baro_f: per-replica box, scaled by e^(2 b h) per BAOA
    float *ke;                     // nullable: per-atom kinetic energy m v^2 / 2 (kcal/mol) after the update
    // nullable: the fast force before its mean subtraction; when set, the
    // force used is fast_pre minus the replica mean formed from fast_sum (the
    // exact fixed-point sums of launch_nc_convert) and it is written to
    // fast_out (f_fast is then not read)
    const float *fast_pre;
    const unsigned long long *fast_sum;
    float *fast_out;
};
void launch_integrate(const IntegArgs &a, cudaStream_t st);

// Per-replica FP64 kinetic energy, total energy and kinetic temperature of a
// state whose velocities still lack the closing kicks selected here.
struct ThermoArgs {
    const int *rep_off;
    const float *v, *f_fast, *f_slow, *masses;
    float h_in, h_out;
    int close_b, kick_l;           // apply v += h_in a F_fast, then v += h_out a (F_slow - F_fast)
    const unsigned long long *fast_sum;   // nullable: [R][3] fixed-point sums whose mean is still to be
                                          // subtracted from f_fast
    const double *energy;          // [R] potential energy U at the same configuration
    double *out;                   // [R][3]: K, U + K, T
    double *trace;                 // nullable: [R][3] copy (one row of a per-outer-step trace)
    const int *part_off;           // [R+1] replica-local parts (launch_mean_part_off)
    double *partial;               // scratch of thermo_scratch_bytes(n_atoms, n_rep) bytes
    int n_rep;
};
size_t thermo_scratch_bytes(int n_atoms, int n_rep);
void launch_thermo(const ThermoArgs &a, int n_atoms, int n_rep, cudaStream_t st);

// Barostat of the outer step (piston on epsilon = ln(V)/3; see dmts_integrator).
struct BaroArgs {
    int n_rep;
    const int *rep_off;
    double *baro;                  // [R][3]: p_eps, G, flag
    float *box;                    // [R][3]
    const double *K;               // [R] kinetic energy (kcal/mol)
    const double *wvir;            // [R] virial: the estimator (end) or the full force's (first start)
    float *baro_f;                 // [R][3] out (start): the A half-step factors
    const uint64_t *seed;
    const uint32_t *rep_id;
    const uint64_t *step;
    uint64_t step_add;
    double delta_outer, h, p_kcal, tau_fs, kT;
    const int *err;
};
// start of an outer step: G (when unset), half kick, Ornstein-Uhlenbeck step, factors
void launch_baro_start(const BaroArgs &a, cudaStream_t st);
// end of an outer step: G from K and the estimator, half kick
void launch_baro_end(const BaroArgs &a, cudaStream_t st);
void launch_advance_step(uint64_t *step, int n_rep, uint64_t add, const int *err, cudaStream_t st);
void launch_embed(int n, int C, const uint8_t *species, const float *emb, float *s, cudaStream_t st);
void launch_rowsum(int n, int C, const float *u, float scale, float *e_atom, cudaStream_t st);

}  // namespace dmts
