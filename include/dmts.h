/*
 * dmts.h -- C ABI of the GB300 (sm_103a) DMTS-NC library.
 *
 * The library runs one dual-level RESPA molecular-dynamics step (Algorithm 1
 * of the paper, "DMTS-NC Integration Step"): an expensive conservative
 * message-passing potential U, with forces F = -grad U (Sec. 2, "Multi-time-
 * step integrator"), is evaluated once per outer step Delta; a cheap
 * non-conservative direct-force model F_NC (Sec. 2, "Model architecture") is
 * evaluated at each of the n inner steps delta = Delta/n. The inner steps are
 * BAOAB steps (Sec. 2, B-A-O-A-B splitting) whose O-part is a Langevin
 * thermostat with species-dependent friction (Sec. 2, "High Hydrogen
 * Friction"); masses follow hydrogen mass repartitioning (Sec. 2, "HMR").
 *
 * Conventions shared by every call
 *  - Units: Angstrom, femtosecond, amu, kcal/mol, kelvin.
 *  - Pointers documented as "device" are CUDA device pointers on the
 *    context's device, owned by the caller; "host" pointers are ordinary host
 *    memory, also owned by the caller. The library owns only its internal
 *    workspace (weights, neighbour-list scratch, activations), released by
 *    dmts_destroy / dmts_state_release.
 *  - Arrays are contiguous, row-major: positions/velocities/forces are float
 *    [n_atoms][3]; species are uint8 codes 0..n_species-1 (H must be 0).
 *  - Several replicas (independent systems) may be batched in one call: atoms
 *    of replica r occupy [rep_off[r], rep_off[r+1]). Replicas never interact.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Calls only
 *    enqueue work, except where noted ("synchronous").
 *  - Errors: every call returns a dmts_status; dmts_last_error() gives text.
 *    Argument errors are reported before any work is enqueued and leave all
 *    outputs untouched. Device-detected errors (neighbour-list overflow,
 *    non-finite positions) are recorded in a sticky device word; from then on
 *    kernels of this context skip their updates, and dmts_sync() returns the
 *    error. Outputs of the failed call are then unspecified.
 */
#ifndef DMTS_H
#define DMTS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DMTS_MAX_SPECIES 8
#define DMTS_MAX_LAYERS 4

typedef enum {
    DMTS_OK = 0,
    DMTS_E_INVALID = 1,       /* bad argument or unsupported model size */
    DMTS_E_OOM = 2,           /* device allocation failed */
    DMTS_E_CUDA = 3,          /* a CUDA call failed */
    DMTS_E_NBR_OVERFLOW = 4,  /* neighbour list larger than its capacity */
    DMTS_E_NONFINITE = 5,     /* NaN/Inf found in positions or velocities */
    DMTS_E_TIMEOUT = 6,       /* a bounded wait of a device kernel on its own asynchronous copies or
                                 tensor-core work gave up; the context stays usable */
    DMTS_E_BUSY = 7           /* state already in use by an unfinished call */
} dmts_status;

/*
 * Arithmetic of the MLP contractions, and of the per-edge radial
 * contraction R_lc = sum_k W_lkc f_c B_k of a conservative model with
 * C = 128 (the paper states none; the stand-in models run them as
 * follows). DMTS_FP32: fp32 SIMT products. DMTS_BF16:
 * tensor cores, bf16 x bf16 products accumulated in fp32, each operand held
 * as a split pair hi = rn_bf16(v), lo = rn_bf16(v - hi) and the products
 * hi*hi + lo*hi + hi*lo accumulated (about 16 significant bits per operand;
 * forces within 2e-3 of the model force's RMS). DMTS_BF16_PLAIN: the same
 * kernels with the hi*hi products only (one bf16 rounding per operand,
 * a third of the tensor-core work; forces off by a few per cent of the
 * message-passing force's RMS).
 */
typedef enum { DMTS_FP32 = 0, DMTS_BF16 = 1, DMTS_BF16_PLAIN = 2 } dmts_precision;

/*
 * Message-passing model (both the conservative model and the embedding of
 * the NC model are built from the same layer; Sec. 2 "Model architecture").
 *
 * Layer t, for every receiver i and neighbour j within rc (r = |x_j - x_i|,
 * minimum image, n = (x_j - x_i)/r):
 *   B_k(r)   = sqrt(2/rc) sin(k pi r/rc)/r, k = 1..K   (Bessel basis)
 *   f(u)     = 1 - (p+1)(p+2)/2 u^p + p(p+2) u^(p+1) - p(p+1)/2 u^(p+2), u = r/rc
 *   R_lc(r)  = f(r/rc) sum_k wrad[l][k][c] B_k(r)
 *   A_i[lm][c] = nu sum_j R_lc(r_ij) s_j[c] Y_lm(n_ij)   (real SH, component
 *                normalisation, l <= lmax, order [00 | x y z | xy yz (3z^2-1) xz (x^2-y^2)])
 *   q_i[l*C+c] = sum_m A_i[lm][c]^2
 *   s_i <- s_i + W2 silu(W1 q_i + b1) + b2
 * with s_i^0 = emb[species_i].
 *
 * Conservative model: U_MP = scale * sum_i sum_o wo[o] silu((Wr s_i^L + br)[o]).
 *   Weight blob (float64, host): emb[S][C]; for each layer: wrad[lmax+1][K][C],
 *   W1[C][(lmax+1)C], b1[C], W2[C][C], b2[C]; then Wr[C][C], br[C], wo[C].
 *
 * NC model (one layer, lmax = 1): x_i = s_i^1, V_ih = sum_c U[h][c] A_i[l=1][c]
 * (a 3-vector per tensor head h < n_l), q_ih = Wq[h] x_i, k_ih = Wk[h] x_i
 * (h < H = K + n_l, each in R^n_c), c_ijh = q_ih . k_jh / sqrt(n_c),
 *   F_ij = (sum_{h<K} c_ijh B_{h+1}(r)) (n_ij + sum_{h<n_l} c_ij(K+h) V_ih) f(r/rc),
 *   F_i  = scale * sum_{j in N(i)} (F_ij - F_ji)  (+ bonded prior force),
 * then the replica's FP64 mean force is subtracted from every atom.
 *   Weight blob (float64, host): emb[S][C]; wrad[2][K][C], W1[C][2C], b1[C],
 *   W2[C][C], b2[C]; U[n_l][C]; Wq[H][n_c][C]; Wk[H][n_c][C].
 *
 * Supported sizes: conservative C in {32, 64, 128}, lmax in {0, 1, 2}, K = 8,
 * L <= DMTS_MAX_LAYERS; NC C in {32, 64}, K = 8, n_c = 8, n_l <= 4.
 */
typedef struct {
    int L, C, lmax, K, n_species;
    int n_c, n_l;              /* NC head only (0 for the conservative model) */
    float rc;                  /* cutoff (A) */
    float p_env;               /* envelope exponent p (integer valued, 2..12) */
    float nu;                  /* message normalisation */
    float scale;               /* energy scale (conservative) / force scale (NC) */
    int precision;             /* dmts_precision of the MLP contractions */
    const double *weights;     /* host blob, layout above */
    long long n_weights;       /* number of doubles in the blob (checked) */
} dmts_model;

/*
 * Analytic terms of U besides the message-passing energy U_MP:
 *  - harmonic bonds 1/2 k_bond (r - r0)^2;
 *  - Lennard-Jones 4 eps ((sig/r)^12 - (sig/r)^6) f(r/lj_rc; lj_p) between
 *    heavy atoms (species != 0) of different molecules;
 *  - the screened nuclear repulsion E_rep of Sec. 2 between every pair that
 *    is not bonded: E_rep = k_e Z_i Z_j / r phi(r/a_ij) f(r/rep_rc; rep_p), with
 *    Z = (1, 6, 7, 8, 16) for species codes (H, C, N, O, S), k_e = 332.0637133
 *    kcal/mol A, and the universal screening function of Ziegler, Biersack and
 *    Littmark standing in for the NHL pair parameters the paper cites but does
 *    not give: phi(x) = sum_k c_k exp(-d_k x), c = (0.18175, 0.50986, 0.28022,
 *    0.02817), d = (3.19980, 0.94229, 0.40290, 0.20162),
 *    a_ij = 0.8854 a_0 / (Z_i^0.23 + Z_j^0.23), a_0 = 0.529177210903 A.
 * U = U_MP + bonds + LJ + E_rep. The fast force F_S = F_NC + bonds + F_rep
 * (Sec. 2: F_i = sum_j (F_ij - F_ji) + F_rep,i). rep_rc must not exceed the
 * NC cutoff.
 */
typedef struct {
    float k_bond, lj_eps, lj_sigma, lj_rc, lj_p;
    float rep_rc, rep_p;
} dmts_prior;

/*
 * A batch of n_replicas independent systems (device arrays unless noted).
 * bond_ptr/bond_idx/bond_r0 are a per-atom bond table (CSR, both directions:
 * each bond (a, b) appears in a's and in b's row); dmts_bond_table() builds it
 * on the host from a bond list.
 */
typedef struct {
    int n_atoms, n_replicas;
    const int *rep_off;        /* device int32 [n_replicas+1], rep_off[0] = 0 */
    const float *box;          /* device float [n_replicas][3]; 0 on all axes = open boundary */
    float *x;                  /* device float [n_atoms][3] (updated by respa_step) */
    const uint8_t *species;    /* device uint8 [n_atoms] */
    const int *mol_id;         /* device int32 [n_atoms] */
    const int *bond_ptr;       /* device int32 [n_atoms+1] */
    const int *bond_idx;       /* device int32 [bond_ptr[n_atoms]] */
    const float *bond_r0;      /* device float [bond_ptr[n_atoms]] */
} dmts_system;

/* Full (both-direction) neighbour list in CSR form: row i holds every j != i
 * of i's replica with |d_ij|^2 < r_list^2 (minimum image), in a deterministic
 * order (row order is otherwise unspecified). */
typedef struct {
    int *row_ptr;              /* device int32 [n_atoms+1] */
    int *col;                  /* device int32 [capacity] */
    long long capacity;
    float r_list;              /* cutoff of the stored list, model cutoff + skin */
} dmts_nbr;

typedef struct dmts_ctx dmts_ctx;

/* Creates a context on `device` and uploads both models (weights copied;
 * the host blobs may be freed afterwards). Either model pointer may be NULL
 * if the corresponding calls are not used. Synchronous. */
dmts_status dmts_create(dmts_ctx **out, const dmts_model *cons, const dmts_model *nc,
                        const dmts_prior *prior, int device);
void dmts_destroy(dmts_ctx *ctx);
const char *dmts_last_error(const dmts_ctx *ctx);

/* Waits for `stream`, then returns and clears the sticky device error word
 * (DMTS_OK when none). Synchronous. */
dmts_status dmts_sync(dmts_ctx *ctx, void *stream);

/*
 * Cell-list neighbour build (Sec. 2: N(i) = atoms j != i within the cutoff;
 * minimum image for periodic axes). Writes nbr->row_ptr and nbr->col for
 * the list cutoff nbr->r_list. Synchronous: *n_pairs receives the number of
 * stored pairs; if it exceeds nbr->capacity, col is left unspecified and
 * DMTS_E_NBR_OVERFLOW is returned (retry with capacity >= *n_pairs).
 * Periodic boxes need r_list < box/2 on every periodic axis.
 */
dmts_status nbr_build(dmts_ctx *ctx, const dmts_system *sys, dmts_nbr *nbr,
                      long long *n_pairs, void *stream);

/*
 * nbr_build for callers that cannot allocate device memory -- code running
 * where cudaMalloc is unavailable or forbidden (inside a memory-pool-managed
 * framework that owns every device allocation, or in a plug-in that may only
 * touch buffers its host hands it), and callers that have no dmts_ctx
 * because creating one allocates. The paper has no
 * counterpart; this is the same cell-list neighbour build as nbr_build, with
 * identical output.
 *
 * All scratch (cell grid, cell counts and offsets, per-atom cell and slot,
 * per-row counts, replica map, pair total, error word) lives in one static
 * device array of about 3.4 MB that every GPU loading this library keeps
 * until the process exits. Limits: at most DMTS_STATIC_MAX_ATOMS atoms,
 * DMTS_STATIC_MAX_REPLICAS replicas and DMTS_STATIC_MAX_CELLS cells in
 * total; larger inputs are rejected with DMTS_E_INVALID before any device
 * work. The caller passes the system and the list buffers (nbr->row_ptr,
 * nbr->col) as for nbr_build. Works on the current CUDA device; the first
 * call on a device looks up the array's device address, so make that first
 * call before any stream capture. Every call reuses the same array: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller. No cudaMalloc, cudaFree or allocating library
 * routine is called. Synchronous; errors as for nbr_build (the message is
 * read with dmts_last_error(NULL)).
 */
#define DMTS_STATIC_MAX_ATOMS 131072
#define DMTS_STATIC_MAX_CELLS 65536
#define DMTS_STATIC_MAX_REPLICAS 1024
dmts_status nbr_build_noalloc(const dmts_system *sys, dmts_nbr *nbr, long long *n_pairs, void *stream);

#define DMTS_WITH_PRIOR 1      /* energy_forces_cons: add bonds + LJ + E_rep */
#define DMTS_WITH_BONDS 1      /* forces_nc: add the bond forces and F_rep */

/*
 * Conservative energy and forces F = -grad U (Sec. 2, F = -grad U; Algorithm
 * 1, FENNIX_large). energy: device double [n_replicas] (FP64 per-replica sum,
 * may be NULL); forces: device float [n_atoms][3] (may be NULL for energy
 * only). nbr must hold a list with r_list >= model rc (and >= lj_rc with
 * DMTS_WITH_PRIOR), built for the current positions. The forces are the
 * hand-written adjoint of the energy with per-layer recomputation of all
 * edge quantities; only node features are stored. Each pair's force is
 * formed once and added to its two atoms in 32.32 fixed point, so the forces
 * do not depend on the order of the additions (the same bits alone or
 * batched); a pair term that is not finite or exceeds 2^24 in magnitude
 * sets DMTS_E_NONFINITE. virial: device double
 * [n_replicas] (may be NULL; needs forces): -sum_i F_i . q_i in pair form,
 * sum over directed edges of dU/dd_ij . d_ij plus the analytic pair terms
 * (Sec. 2 "Computation of the virial term in NPT": the estimator at the
 * end of an outer step).
 */
dmts_status energy_forces_cons(dmts_ctx *ctx, const dmts_system *sys, const dmts_nbr *nbr,
                               double *energy, float *forces, double *virial, int flags, void *stream);

/*
 * Non-conservative direct forces (Sec. 2 "Model architecture"; Algorithm 1,
 * FENNIX_NC). forces: device float [n_atoms][3]; net_force: device double
 * [n_replicas][3], the per-replica sum before the mean subtraction (may be
 * NULL); virial: device double [n_replicas] (may be NULL), the proxy
 * -sum_i F_i . q_i of Sec. 2 "Computation of the virial term in NPT" in its
 * pair form sum_i sum_{j in N(i)} (F_ij + F_pair,ij / 2) . r_ij, F_pair the
 * repulsion and (with DMTS_WITH_BONDS) bond pair forces. nbr: list with
 * r_list >= NC rc.
 */
dmts_status forces_nc(dmts_ctx *ctx, const dmts_system *sys, const dmts_nbr *nbr,
                      float *forces, double *net_force, double *virial, int flags, void *stream);

typedef enum { DMTS_MODE_RESPA = 0, DMTS_MODE_STS = 1 } dmts_mode;

/* Thermostat of the O-step (Sec. 2, "High Hydrogen Friction"): Langevin, or
 * Fast Forward Langevin, which gives each atom the speed of the Langevin
 * update w = c1 v + c2 sqrt(1/m) G but keeps the direction of v:
 * v <- |w| v / |v| (per-atom 3-vector norms; an atom at rest takes w). */
typedef enum { DMTS_LANGEVIN = 0, DMTS_FFL = 1 } dmts_thermostat;

/*
 * Integrator parameters. RESPA: outer step Delta = dt_outer, n_inner inner
 * BAOAB steps of delta = Delta/n_inner driven by F_S = F_NC (+ bonds), outer
 * kicks by F_L = F - F_S (Algorithm 1). STS: BAOAB with F = -grad U and step
 * dt_outer (n_inner ignored). gamma_ps: Langevin friction per species (1/ps);
 * the O-step is v <- c1 v + c2 sqrt(1/m) G with c1 = exp(-gamma delta),
 * c2 = sqrt((1 - c1^2) kB T), kB T in amu A^2/fs^2.
 */
typedef struct {
    float dt_outer;
    int n_inner;
    float temperature;
    double gamma_ps[DMTS_MAX_SPECIES];
    int mode;                  /* dmts_mode */
    float skin;                /* neighbour-list skin (A); lists rebuilt when an atom moved > skin/2 */
    int thermostat;            /* dmts_thermostat */
    /* Barostat (RESPA mode, periodic replicas; Sec. 3: Bussi's barostat, target
     * pressure and volume relaxation time), read as an isotropic Langevin
     * piston on epsilon = ln(V)/3 with mass W = (N_f + 3) kB T tau_P^2
     * (N_f = 3 n), friction 1/tau_P and matching noise, coupled to the atoms
     * as in the Martyna-Tobias-Klein equations and driven by the virial
     * estimator of Sec. 2 "Computation of the virial term in NPT". Per outer
     * step: p_eps += Delta/2 G; p_eps <- c p_eps + sqrt((1 - c^2) W kB T) xi
     * (c = exp(-Delta/tau_P), xi the first Gaussian of Philox at (seed,
     * replica, step, atom slot 2^32 - 1)); every A half-step h of the outer
     * step moves x <- x e^(b h) + h (e^(b h) - 1)/(b h) v, v <- v e^(-a h),
     * box <- box e^(b h) (b = p_eps/W, a = (1 + 3/N_f) b); at the step's end
     * G = (1 + 3/N_f) 2K - W_est - 3 V P and p_eps += Delta/2 G. The box of
     * each replica (dmts_system.box) is updated in place. Needs st->baro and
     * the three virial arrays of the state. */
    int barostat;              /* 0 off, 1 on */
    float pressure_atm;        /* target pressure (atm) */
    float tau_p_ps;            /* volume relaxation time tau_P (ps) */
} dmts_integrator;

/*
 * Dynamic state of a batch of replicas (device arrays unless noted). The
 * noise of atom i (index within its replica) at inner step s of replica r is
 * Philox4x32-10 with key (seed_lo, seed_hi) and counter
 * (i, replica_id[r], s_lo, s_hi); s counts inner steps (RESPA) or steps (STS).
 */
typedef struct {
    dmts_system sys;
    float *v;                  /* device float [n_atoms][3] (A/fs) */
    float *f_nc;               /* device float [n_atoms][3] cached fast force */
    float *f_cons;             /* device float [n_atoms][3] cached full force */
    const float *masses;       /* device float [n_atoms] simulation masses (amu) */
    double *energy;            /* device double [n_replicas] last potential energy (may be NULL) */
    uint64_t *step;            /* device uint64 [n_replicas] inner-step counters */
    const uint64_t *seed;      /* device uint64 [n_replicas] */
    const uint32_t *replica_id;/* device uint32 [n_replicas] */
    int first_step;            /* host flag: 1 = forces not yet evaluated */
    void *internal;            /* library-owned; NULL before the first call */
    double *virial_nc;         /* device double [n_replicas] (may be NULL): RESPA only, after each outer
                                  step the average over its n inner steps of the fast force's virial
                                  proxy (see forces_nc; Sec. 2 "Computation of the virial term in NPT") */
    double *virial_cons;       /* device double [n_replicas] (may be NULL): virial of the full force
                                  -grad U at the last evaluation (see energy_forces_cons) */
    double *virial_est;        /* device double [n_replicas] (may be NULL; needs virial_cons and, in RESPA
                                  mode, virial_nc): after each outer step the virial estimator of Sec. 2
                                  "Computation of the virial term in NPT": the full force's virial at the
                                  end of the outer step with the fast force's share at that configuration
                                  replaced by its average over the inner steps,
                                  virial_cons - W_NC(q_end) + virial_nc; in STS mode virial_cons */
    double *baro;              /* device double [n_replicas][3] (may be NULL unless the barostat is on):
                                  p_eps (kcal/mol fs), the piston force G at the last step end, and a
                                  flag (1 once G is set; start from zeros) */
    double *thermo;            /* device double [n_replicas][3] (may be NULL; needs energy): at the end of each
                                  call, for the end of its last outer step (velocities after the closing
                                  kicks): the kinetic energy K = sum_i m_i |v_i|^2 / 2 (kcal/mol), the total
                                  energy U + K with U as in `energy`, and the kinetic temperature
                                  2K / (3 n_r kB) (K) of Sec. 3's temperature checks; every per-atom term is
                                  formed in FP64 from the fp32 state and summed in FP64, in an order that
                                  does not depend on the other replicas of the batch */
    double *thermo_trace;      /* device double [thermo_trace_rows][n_replicas][3] (may be NULL; needs thermo):
                                  row o receives the same three values after outer step o of each call */
    int thermo_trace_rows;     /* rows of thermo_trace; a call with more outer steps is rejected */
} dmts_state;

/*
 * Advances every replica of `st` by n_outer outer steps of Algorithm 1
 * (RESPA mode) or n_outer single time steps (STS mode). Forces are cached
 * across calls (first_step). Neighbour lists live in st->internal and are
 * rebuilt on the device when needed. Asynchronous: errors detected on the
 * device surface in dmts_sync(). Ordered after everything already queued on
 * `stream`, and work queued on `stream` afterwards waits for it. In a call
 * of three or more outer steps the second is captured into a CUDA graph and
 * the later ones replay it; a call of one or two outer steps is replayed
 * from a graph kept in st->internal, recaptured whenever the integrator's
 * parameters, the number of steps, an array pointer of `st` or any of the
 * library's device buffers changed (graphs run on a stream of the context,
 * joined to `stream` by events). Should a capture or its instantiation
 * fail, the call runs its launches directly and the context does so from
 * then on. The step counters st->step advance by n_inner (1 in STS mode) at
 * the end of every outer step. The environment variable DMTS_CUDA_GRAPHS=0
 * launches every kernel directly instead (the same kernels and results).
 */
dmts_status respa_step(dmts_ctx *ctx, dmts_state *st, const dmts_integrator *p, int n_outer,
                       void *stream);

/* Frees st->internal. */
void dmts_state_release(dmts_ctx *ctx, dmts_state *st);

/*
 * One step of on-box distillation of the NC model toward target forces (the
 * NC model is a distilled version of the large model trained on forces the
 * large model labels, Sec. 2 "Model training"; its weights, Sec. 2 "Model
 * architecture").
 * Fitted weights (`params`, a mask): DMTS_FIT_QK the head's q/k projection
 * W_qk ([2 H n_c][C]); DMTS_FIT_MLP the channel-mixing MLP of its layer
 * (W1, b1, W2, b2); DMTS_FIT_LAYER the message-passing layer's radial
 * weights W_rad and the tensor-head mix U (the species embedding is not
 * fitted). With F_S the fast force of forces_nc (with
 * DMTS_WITH_BONDS: bonds and repulsion included, mean subtracted) on `sys`
 * and target T (device float [n_atoms][3], e.g. -grad U of the conservative
 * model at the same positions): loss (device double [n_replicas], may be
 * NULL) receives L = sum_i |F_S,i - T_i|^2 per replica; the gradient of
 * sum_r L (the adjoint of the mean subtraction, of the NC head with respect to
 * its q/k rows and V, of the contractions and the MLP, and of the layer with
 * respect to its weights) is written to grad
 * (device float, the length and layout of the NC weight blob, may be NULL),
 * zero for weights not fitted; with lr > 0 one Adam step (beta1 0.9, beta2
 * 0.999, eps 1e-8; adam_step = 1, 2, ... the update count, 1 resets the
 * moments) updates the fitted weights of the context's NC model and their
 * bf16 copies. nbr: the NC list, cutoff >= r_NC. Asynchronous.
 */
#define DMTS_FIT_QK 1
#define DMTS_FIT_MLP 2
#define DMTS_FIT_LAYER 4
dmts_status nc_distill_step(dmts_ctx *ctx, const dmts_system *sys, const dmts_nbr *nbr, const float *target,
                            int params, float lr, int adam_step, double *loss, float *grad, void *stream);

/*
 * Copy of the neighbour list a state holds (inspection; synchronous):
 * which = 0 the conservative list (cutoff r_c + skin), 1 the NC list
 * (r_NC + skin), as last built on the device (Sec. 2, neighbour lists of the
 * two models). row_ptr: device int32 [n_atoms + 1]; col: device int32
 * [col_capacity]; *n_pairs (host) receives the entry count and *r_list (host,
 * may be NULL) the list radius. DMTS_E_INVALID before the state's first
 * respa_step or for a list the state does not hold; DMTS_E_NBR_OVERFLOW with
 * *n_pairs set when col_capacity is too small (row_ptr is written).
 */
dmts_status dmts_state_lists(dmts_ctx *ctx, const dmts_state *st, int which, int32_t *row_ptr, int32_t *col,
                             int64_t col_capacity, int64_t *n_pairs, float *r_list, void *stream);

/* ------------------------------------------------------------------ rewind */
/*
 * Guard against rare disagreements of the two force models (Sec. 2,
 * "Preventing rare model disagreements (Rewind procedure)"): the run is cut
 * into chunks of chunk_outer outer steps with a saved frame at the start of
 * each. If, during a chunk, max |F - F_S| of any replica exceeds
 * `threshold` (kcal/mol/A; measured at every outer kick) or a position or
 * velocity became non-finite, the whole batch goes back to the saved frame
 * and runs sts_steps single-time-step BAOAB steps of sts_dt (the same
 * temperature, frictions, thermostat and skin, the full force -grad U),
 * then resumes Algorithm 1 from there with fresh force caches.
 * sts_steps * sts_dt must be a whole number m >= 1 of outer steps: the STS
 * segment counts as m outer steps of the n_outer requested. Noise counters
 * restart from the saved frame's, so a replayed segment is the same STS
 * trajectory a direct STS run from the frame gives, bit for bit.
 */
typedef struct {
    float threshold;           /* kcal/mol/A; +inf disables the force check */
    int chunk_outer;           /* outer steps between saved frames (>= 1) */
    int sts_steps;             /* STS steps after a rewind (>= 1) */
    float sts_dt;              /* STS time step (fs) */
} dmts_guard;

typedef struct {
    int n_rewinds;             /* out */
    int n_chunks;              /* out: chunks of Algorithm 1 attempted */
    float *chunk_max;          /* host [chunk_cap] (may be NULL): max |F - F_S| of each chunk */
    int chunk_cap;
    float *rewind_at;          /* host [rewind_cap] (may be NULL): outer steps completed at each rewind */
    int rewind_cap;
} dmts_guard_stats;

/* n_outer outer steps of Algorithm 1 on `st` (p->mode must be RESPA) under
 * the rewind guard. Allocates its saved frame per call (device: x, v, F_NC
 * and the full force, four [N][3] float arrays, the per-replica step
 * counters and energies and, with the barostat, the boxes and piston
 * states); synchronises the stream once per chunk to read the monitor. Returns DMTS_E_NONFINITE if the STS segment
 * itself goes non-finite, DMTS_E_INVALID for bad parameters. */
dmts_status respa_guarded(dmts_ctx *ctx, dmts_state *st, const dmts_integrator *p, const dmts_guard *guard,
                          int n_outer, dmts_guard_stats *stats, void *stream);

/* ------------------------------------------------------------------ serving */

typedef struct {
    int n_atoms;
    const float *x;            /* host [n_atoms][3] */
    const float *v;            /* host [n_atoms][3] */
    const uint8_t *species;    /* host [n_atoms] */
    const int *mol_id;         /* host [n_atoms] */
    int n_bonds;
    const int *bonds;          /* host [n_bonds][2] */
    const float *bond_r0;      /* host [n_bonds] */
    const float *masses;       /* host [n_atoms] simulation masses */
    float box[3];              /* 0 = open boundary */
    int n_outer;               /* outer steps to run */
    uint64_t seed;
    uint32_t replica_id;
    double arrival_s;          /* arrival time relative to the start of the run */
} dmts_request;

typedef struct {
    long long hbm_budget_bytes;   /* admission limit on the device footprint */
    int max_slots;                /* at most this many replicas resident */
    int realtime;                 /* 1: admit a request only after its arrival time */
} dmts_serve_cfg;

typedef struct {
    float *x, *v;              /* host [n_atoms][3], filled on completion */
    double energy;             /* last potential energy */
    double t_arrival_s, t_admit_s, t_done_s;
    int status;                /* dmts_status of this request */
} dmts_result;

typedef struct {
    double *tick_ms;           /* host array of capacity tick_cap (may be NULL) */
    int tick_cap;
    int n_ticks;               /* out */
    double wall_s;             /* out: duration of the whole run */
    double atom_outer_steps;   /* out: sum over ticks of resident atoms */
    int max_resident;          /* out */
    int *tick_atoms;           /* host array of capacity tick_cap (may be NULL): atoms in the packed batch
                                  each tick integrated (resident replicas, and retired ones not yet
                                  removed by a re-pack) */
} dmts_serve_stats;

/*
 * Continuous-batching serving loop: requests are admitted in arrival order
 * while the slot count and the HBM budget allow; every tick runs one batched
 * outer step (one launch sequence over all resident replicas); finished
 * replicas are copied back and retired, freeing room for waiting ones.
 * Synchronous.
 */
dmts_status run_replicas(dmts_ctx *ctx, const dmts_request *reqs, int n_req,
                         const dmts_integrator *p, const dmts_serve_cfg *cfg,
                         dmts_result *out, dmts_serve_stats *stats);

/* --------------------------------------------------------- host helpers */

/* Hydrogen mass repartitioning (Sec. 2 "HMR"): every H (species 0) gains
 * delta_h; each molecule's total gain is removed from its heavy atoms in
 * proportion to their masses, so molecular masses are preserved. Host, FP64. */
void dmts_masses_hmr(int n_atoms, const uint8_t *species, const int *mol_id,
                     const double *masses_in, double delta_h, double *masses_out);

/* Per-atom bond table (CSR, both directions) from a bond list. bond_ptr has
 * n_atoms+1 entries, bond_idx and bond_r0_out 2*n_bonds. Host. */
dmts_status dmts_bond_table(int n_atoms, int n_bonds, const int *bonds, const float *bond_r0,
                            int *bond_ptr, int *bond_idx, float *bond_r0_out);

/* Philox4x32-10 noise words for testing: out[4*i..4*i+3] = Philox(key =
 * (seed_lo, seed_hi), counter = (atom0 + i, replica, step_lo, step_hi)), i <
 * count. out: device uint32 [4*count]. */
dmts_status dmts_philox_words(dmts_ctx *ctx, uint64_t seed, uint32_t replica, uint64_t step,
                              uint32_t atom0, int count, uint32_t *out, void *stream);

/* The three Gaussians the O-step draws for the same counters. out: device
 * float [3*count]. */
dmts_status dmts_gaussians(dmts_ctx *ctx, uint64_t seed, uint32_t replica, uint64_t step,
                           uint32_t atom0, int count, float *out, void *stream);

/* One channel-mixing contraction as the MLPs run it in bf16 mode (Sec. 2
 * "Model architecture": the perceptrons of both models): out[M][N] =
 * act[M][K] x wt[N][K]^T on the tensor cores, bf16 operands, fp32
 * accumulation. split = 0: act is bf16 [M][K] and wt bf16 [N][K].
 * split = 1: both are split pairs, act [M][2K] and wt [N][2K], each row
 * holding the hi parts in columns [0, K) and the lo parts in [K, 2K), and
 * out = act_hi wt_hi^T + act_lo wt_hi^T + act_hi wt_lo^T (DMTS_BF16).
 * Device pointers, row-major, 16-byte aligned; K a multiple of 64, N a
 * multiple of 16, M >= 1, else DMTS_E_INVALID. */
dmts_status dmts_contract_bf16(dmts_ctx *ctx, int M, int N, int K, const void *act_bf16, const void *wt_bf16,
                               float *out, int split, void *stream);

/* (No counterpart in the paper: failure detection.) Exercises the bounded
 * waits every kernel of this library uses on its mbarriers: launches one
 * block that waits, with that same wait but a limit of limit_us
 * microseconds, on an mbarrier of its own shared memory on which nothing
 * ever arrives and which no copy targets. The wait runs out, the block
 * records DMTS_E_TIMEOUT in the context's sticky error word and returns; the
 * next dmts_sync() returns DMTS_E_TIMEOUT (and clears it) and the context
 * stays usable. limit_us in [1, 1000000], else DMTS_E_INVALID. */
dmts_status dmts_check_bounded_wait(dmts_ctx *ctx, int limit_us, void *stream);

/* Bytes of device workspace a replica of n_atoms needs in the serving loop
 * (admission accounting). */
long long dmts_replica_footprint(const dmts_ctx *ctx, int n_atoms);

/* ------------------------------------------------------ instrumentation */
/* (No counterpart in the paper: measurement support.) While enabled, every
 * named step of the context (one kernel, or a few that always run together,
 * such as the cell pass of the neighbour build) is bracketed by a pair of
 * CUDA events on its own stream. dmts_profile_read() synchronises the device
 * and returns, for slot `idx` (0 <= idx < count returned by a call with
 * idx = -1), the step's name, number of executions and summed duration in ms
 * since the last enable. Disabling clears nothing; enabling clears the table.
 * enable = N > 1 times, inside respa_step and respa_guarded, only every N-th
 * outer step counted from the enable (outer steps 0, N, 2N, ...), so that the
 * events perturb a long run less; other calls are always timed. */
dmts_status dmts_profile_enable(dmts_ctx *ctx, int enable);
int dmts_profile_read(dmts_ctx *ctx, int idx, char *name, int name_cap, long long *launches,
                      double *total_ms);

/* (No counterpart in the paper: measurement support.) Number of kernels this
 * library has launched in this process since it was loaded, over all
 * contexts and devices (counted on the host at each launch). The difference
 * of two reads around a region is the region's launch count. */
unsigned long long dmts_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* DMTS_H */
