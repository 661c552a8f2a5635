// Internal host-side structures of the library.
#pragma once
#include <string>
#include <vector>

#include "common.cuh"
#include "md.cuh"
#include "mp.cuh"
#include "nbr.cuh"

namespace dmts {

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
    bool ensure(size_t bytes);
    void release();
};
// Counts the library's device (re)allocations and frees: a captured graph
// recorded with an older value may hold pointers that are no longer valid.
unsigned long long alloc_generation();
void bump_alloc_generation();

struct DevModel {
    int L = 0, C = 0, lmax = 0, K = 0, S = 0, nc = 0, nl = 0, p = 0;
    float rc = 0.f, nu = 0.f, scale = 0.f;
    bool bf16 = false;                    // MLP contractions on the tensor cores
    int nseg = 1;                         // 3: split-bf16 products (hi*hi + lo*hi + hi*lo); 1: hi*hi only
    float *dev = nullptr;                 // one allocation holding every tensor (the blob's order)
    size_t n_weights = 0;                 // floats in that allocation
    float *emb = nullptr;
    float *wrad[DMTS_MAX_LAYERS] = {}, *w1[DMTS_MAX_LAYERS] = {}, *b1[DMTS_MAX_LAYERS] = {},
          *w2[DMTS_MAX_LAYERS] = {}, *b2[DMTS_MAX_LAYERS] = {};
    float *wr = nullptr, *br = nullptr, *wo = nullptr;
    float *U = nullptr, *Wqk = nullptr;
    // split-bf16 copies for the tensor-core contractions, every one K-major
    // ([out][2 in]: hi | lo): W1, W2, Wr (forward), their transposes
    // (adjoint), Wqk.
    __nv_bfloat16 *dev_bf = nullptr;
    __nv_bfloat16 *w1_bf[DMTS_MAX_LAYERS] = {}, *w2_bf[DMTS_MAX_LAYERS] = {}, *w1t_bf[DMTS_MAX_LAYERS] = {},
                  *w2t_bf[DMTS_MAX_LAYERS] = {};
    __nv_bfloat16 *wr_bf = nullptr, *wrt_bf = nullptr, *wqk_bf = nullptr;
};

constexpr int kNbrSlots = 128;   // longest row kept by the count pass of a state's rebuild

struct NbrScratch {
    Buf grid, cell_cnt, cell_start, cell_atoms, atom_cell, atom_slot, counts, total, counts_sub;
    Buf slots;    // [n_atoms][kNbrSlots] sorted rows kept between the count and the fill of a rebuild
    Buf scan;     // prefix-scan status words [2][scan_tiles] and epoch/tile counters [2] (zero-initialised)
    int scan_tiles = 0;
    void release_all() {
        grid.release(); cell_cnt.release(); cell_start.release(); cell_atoms.release();
        atom_cell.release(); atom_slot.release(); counts.release(); total.release(); counts_sub.release();
        slots.release(); scan.release();
        scan_tiles = 0;
    }
};

struct Workspace {
    Buf s, A, q, h, act, u, gz, gs0, gs1, gA, e_atom, ftmp, atom_rep;
    Buf nc_s, nc_q, nc_act, nc_qk, nc_v, nc_f;
    Buf nc_ffix;      // NC head forces in 32.32 fixed point, zero between evaluations
    Buf nc_next;      // the NC head's work counter, zero between evaluations
    Buf nc_sum;       // per-replica exact sums of the NC forces (fixed point) of the last evaluation
    // split-bf16 operands of the tensor-core contractions ([rows][2K])
    Buf q_bf, act_bf, s_bf, gz_bf, gs0_bf, gs1_bf, nc_q_bf, nc_act_bf, nc_s_bf;
    Buf ms_scratch;   // per-part sums of the mean subtraction
    Buf nc_w;         // per-atom virial proxy of the fast force
    Buf cons_w;       // per-atom virial of the conservative force
    Buf cons_ffix, cons_wfix;   // the adjoint's forces and virial in 32.32 fixed point, zero between evaluations
    Buf nc_w_last;    // per-replica fast-force virial of the last inner step
    // distillation of the NC model: residual, q/k-row and feature gradients,
    // pre-activation, blob-shaped weight gradient, Adam moments, split sums
    Buf dist_F, dist_g, dist_sq, dist_gqk, dist_gs1, dist_gh, dist_h, dist_dw, adam_m, adam_v, dist_part;
    Buf dist_A, dist_gq, dist_gv;
    void release_all() {
        Buf *all[] = {&s, &A, &q, &h, &act, &u, &gz, &gs0, &gs1, &gA, &e_atom, &ftmp, &atom_rep,
                      &nc_s, &nc_q, &nc_act, &nc_qk, &nc_v, &nc_f, &nc_ffix, &nc_next, &nc_sum,
                      &q_bf, &act_bf, &s_bf, &gz_bf, &gs0_bf, &gs1_bf, &nc_q_bf, &nc_act_bf, &nc_s_bf,
                      &ms_scratch, &nc_w, &cons_w, &cons_ffix, &cons_wfix, &nc_w_last,
                      &dist_F, &dist_g, &dist_sq, &dist_gqk, &dist_gs1, &dist_gh, &dist_h, &dist_dw,
                      &adam_m, &adam_v, &dist_part, &dist_A, &dist_gq, &dist_gv};
        for (Buf *b : all) b->release();
    }
};

// Device view of a batch used by the force evaluations.
struct SysView {
    int n, n_rep;
    const int *rep_off;
    const float *box;
    const float *x;
    const uint8_t *species;
    const int *mol_id;
    const int *bond_ptr, *bond_idx;
    const float *bond_r0;
    const int *atom_rep;
    const int *order = nullptr;   // processing order of the per-atom kernels (nullable)
    const int *ms_part_off = nullptr;   // mean-subtraction part offsets of this batch (nullable)
};

struct StateInternal {
    int n = 0, n_rep = 0, n_cells = 0;
    float skin = 0.f, r_cons = 0.f, r_nc = 0.f, grid_margin = 0.f;
    std::vector<CellGrid> grids;
    Buf cons_row, cons_col, nc_row, nc_col, x_ref, gate, atom_rep, ms_part;
    Buf baro_ke, baro_K, baro_f;   // barostat: per-atom kinetic energy, per-replica sum, drift factors
    Buf thermo_part;               // per-part FP64 kinetic-energy sums
    long long cons_cap = 0, nc_cap = 0;
    NbrScratch scratch;
    // respa_step's cached graph of a short call and what it depends on
    cudaGraphExec_t call_graph = nullptr;
    std::vector<uint64_t> call_key;
    unsigned long long call_launches = 0;
};

struct ProfSlot {
    std::string name;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    long long launches;
    double ms;
};

struct Profiler {
    bool on = false;
    int every = 1;          // inside respa_step: time every N-th outer step
    long long outer = 0;    // outer steps seen since enabling
    bool active = true;     // timing the current outer step
    std::vector<ProfSlot> slots;
    std::vector<cudaEvent_t> pool;
    int slot(const char *name);
    cudaEvent_t take();
    void flush();
    void clear();
    void release();
};

}  // namespace dmts

struct dmts_ctx;

namespace dmts {
// Brackets the launches issued in its lifetime with CUDA events when the
// context's profiler is on.
struct ProfScope {
    Profiler *p;
    cudaStream_t s;
    int k;
    cudaEvent_t start = nullptr;
    ProfScope(dmts_ctx *ctx, const char *name, cudaStream_t st);
    ~ProfScope();
};
}  // namespace dmts

struct dmts_ctx {
    int device = 0;
    dmts::DevModel cons, nc;
    bool has_cons = false, has_nc = false;
    dmts_prior prior{};
    int *d_err = nullptr;
    std::string last_error;
    dmts::Workspace ws;
    dmts::NbrScratch nbr_scratch;
    dmts::Profiler prof;
    // second stream of respa_step: the NC evaluation at the end of an outer
    // step runs on it, concurrently with the conservative evaluation at the
    // same positions (created on first use)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // stream of respa_step's graph-replayed outer steps (a capturable stream
    // whatever the caller's), joined to the caller's stream by two events
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    bool graphs_off = false;   // a capture or instantiation failed once: launch directly
};

namespace dmts {
bool ck(dmts_ctx *ctx, cudaError_t e, const char *what);
dmts_status fail(dmts_ctx *ctx, dmts_status s, const std::string &msg);
// Internal flag of cons_eval / nc_eval: the layer-0 features (the species
// embedding) already in the workspace belong to this system, so the
// embedding is not recomputed (set within one respa_step call, where the
// species do not change).
constexpr int kFlagEmbedded = 1 << 30;
// Internal flag of nc_eval: keep the layer output A (ws.dist_A) and the MLP
// pre-activation (ws.dist_h) for the distillation's backward pass.
constexpr int kFlagKeepPre = 1 << 29;
// Internal flag of nc_eval (respa_step): leave the mean subtraction to the
// integrator; the force before it stays in ws.nc_f and the replicas' exact
// sums in ws.nc_sum (forces is not written).
constexpr int kFlagDeferMean = 1 << 28;
dmts_status cons_eval(dmts_ctx *ctx, const SysView &s, const int *row_ptr, const int *col, double *energy,
                      float *forces, int flags, cudaStream_t st, double *virial = nullptr);
dmts_status nc_eval(dmts_ctx *ctx, const SysView &s, const int *row_ptr, const int *col, float *forces,
                    double *net, int flags, cudaStream_t st, double *virial = nullptr, int virial_accumulate = 0);
// grid_margin: periodic cell edges are at least r_list (1 + grid_margin), so
// that the box may shrink by that fraction (a barostat) before a rebuild fails.
dmts_status setup_grids(dmts_ctx *ctx, const std::vector<int> &rep_off, const std::vector<float> &box,
                        float r_list, std::vector<CellGrid> &grids, int &n_cells, float grid_margin = 0.f);
SysView state_view(dmts_state *stt);
RepTable rep_table(const dmts_ctx *ctx);
void rebuild_lists(dmts_ctx *ctx, StateInternal *si, const SysView &v, cudaStream_t st);
void state_force_rebuild(dmts_ctx *ctx, dmts_state *stt, cudaStream_t st);
// cache_short_calls: a call of one or two outer steps may be replayed from
// the state's cached graph (respa_step; not the serving loop, whose packed
// batch changes from tick to tick)
dmts_status respa_run(dmts_ctx *ctx, dmts_state *stt, const dmts_integrator *p, int n_outer, cudaStream_t st,
                      unsigned *fl_max, bool cache_short_calls = false);
void prepare_nbr_work_async(dmts_ctx *ctx, StateInternal *si, const SysView &v, NbrWork &nw);
}  // namespace dmts

// (Re)initialises st->internal for the current shape of st->sys, re-using
// its buffers when present; leaves the lists built for the current positions.
dmts_status init_state(dmts_ctx *ctx, dmts_state *stt, float skin, cudaStream_t st, float grid_margin = 0.f);
// Cell margin of states integrated with the barostat: the box may shrink by
// this fraction before a list rebuild reports DMTS_E_INVALID.
constexpr float kBaroGridMargin = 0.05f;
void free_state_internal(dmts::StateInternal *si);
