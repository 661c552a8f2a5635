// Continuous-batching serving loop over independent MD replicas.
//
// Resident replicas are packed into one batch (atoms concatenated, ragged
// replica offsets) and advanced together, one outer step of Algorithm 1 per
// tick, by the same launch sequence as respa_step. Requests are admitted in
// arrival order while the slot count and the device-memory budget allow;
// their first forces are evaluated in a separate admission batch and their
// state is then spliced into the packed batch. Finished replicas are copied
// back at once and leave the batch at the next re-pack, which happens at most
// every kRepackTicks ticks (or at once when the batch is idle).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "engine.cuh"

using namespace dmts;

namespace {

constexpr int kRepackTicks = 4;

struct Packed {
    Buf x, v, fnc, fcons, masses, species, mol, bptr, bidx, br0, rep_off, box, seed, rid, step, energy;
    void release() {
        Buf *all[] = {&x, &v, &fnc, &fcons, &masses, &species, &mol, &bptr, &bidx, &br0, &rep_off, &box,
                      &seed, &rid, &step, &energy};
        for (Buf *b : all) b->release();
    }
};

struct Slot {
    int req;
    int n;
    int done;          // outer steps completed
    bool finished;     // results copied out; leaves at the next re-pack
};

__global__ void k_gather_state(int n, const int *map, const float *x0, const float *v0, const float *a0,
                               const float *b0, float *x1, float *v1, float *a1, float *b1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = map[i];
    if (j < 0) return;
    for (int c = 0; c < 3; ++c) {
        x1[3 * i + c] = x0[3 * j + c];
        v1[3 * i + c] = v0[3 * j + c];
        a1[3 * i + c] = a0[3 * j + c];
        b1[3 * i + c] = b0[3 * j + c];
    }
}

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Host image of a batch of requests, uploaded into the static arrays of `pk`.
struct HostBatch {
    std::vector<int> rep_off;
    std::vector<float> box, masses;
    std::vector<uint8_t> species;
    std::vector<int> mol, bptr, bidx;
    std::vector<float> br0;
    std::vector<uint64_t> seed, step;
    std::vector<uint32_t> rid;
};

dmts_status build_host_batch(const dmts_request *reqs, const std::vector<int> &order, const std::vector<uint64_t> &steps,
                             HostBatch &h) {
    h = HostBatch();
    h.rep_off.push_back(0);
    std::vector<int> bonds;
    std::vector<float> r0;
    for (size_t k = 0; k < order.size(); ++k) {
        const dmts_request &q = reqs[order[k]];
        const int off = h.rep_off.back();
        h.rep_off.push_back(off + q.n_atoms);
        for (int a = 0; a < 3; ++a) h.box.push_back(q.box[a]);
        h.masses.insert(h.masses.end(), q.masses, q.masses + q.n_atoms);
        h.species.insert(h.species.end(), q.species, q.species + q.n_atoms);
        h.mol.insert(h.mol.end(), q.mol_id, q.mol_id + q.n_atoms);
        for (int b = 0; b < q.n_bonds; ++b) {
            bonds.push_back(q.bonds[2 * b] + off);
            bonds.push_back(q.bonds[2 * b + 1] + off);
            r0.push_back(q.bond_r0[b]);
        }
        h.seed.push_back(q.seed);
        h.rid.push_back(q.replica_id);
        h.step.push_back(steps[k]);
    }
    const int N = h.rep_off.back();
    const int nb = (int)r0.size();
    h.bptr.assign(N + 1, 0);
    h.bidx.assign(std::max(1, 2 * nb), 0);
    h.br0.assign(std::max(1, 2 * nb), 0.f);
    return dmts_bond_table(N, nb, bonds.data(), r0.data(), h.bptr.data(), h.bidx.data(), h.br0.data());
}

bool upload_static(Packed &pk, const HostBatch &h, cudaStream_t st) {
    const int N = h.rep_off.back(), R = (int)h.rep_off.size() - 1;
    auto up = [&](Buf &b, const void *src, size_t bytes) {
        return b.ensure(std::max<size_t>(bytes, 16)) &&
               (bytes == 0 || cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess);
    };
    return up(pk.rep_off, h.rep_off.data(), sizeof(int) * (R + 1)) && up(pk.box, h.box.data(), sizeof(float) * 3 * R) &&
           up(pk.masses, h.masses.data(), sizeof(float) * N) && up(pk.species, h.species.data(), N) &&
           up(pk.mol, h.mol.data(), sizeof(int) * N) && up(pk.bptr, h.bptr.data(), sizeof(int) * (N + 1)) &&
           up(pk.bidx, h.bidx.data(), sizeof(int) * h.bidx.size()) &&
           up(pk.br0, h.br0.data(), sizeof(float) * h.br0.size()) &&
           up(pk.seed, h.seed.data(), sizeof(uint64_t) * R) && up(pk.rid, h.rid.data(), sizeof(uint32_t) * R) &&
           up(pk.step, h.step.data(), sizeof(uint64_t) * R) && pk.energy.ensure(sizeof(double) * (R + 1)) &&
           pk.x.ensure(sizeof(float) * 3 * (N + 1)) && pk.v.ensure(sizeof(float) * 3 * (N + 1)) &&
           pk.fnc.ensure(sizeof(float) * 3 * (N + 1)) && pk.fcons.ensure(sizeof(float) * 3 * (N + 1));
}

void fill_state(dmts_state &s, Packed &pk, const HostBatch &h) {
    void *internal = s.internal;
    memset(&s, 0, sizeof s);
    s.internal = internal;
    s.sys.n_atoms = h.rep_off.back();
    s.sys.n_replicas = (int)h.rep_off.size() - 1;
    s.sys.rep_off = (const int *)pk.rep_off.p;
    s.sys.box = (const float *)pk.box.p;
    s.sys.x = (float *)pk.x.p;
    s.sys.species = (const uint8_t *)pk.species.p;
    s.sys.mol_id = (const int *)pk.mol.p;
    s.sys.bond_ptr = (const int *)pk.bptr.p;
    s.sys.bond_idx = (const int *)pk.bidx.p;
    s.sys.bond_r0 = (const float *)pk.br0.p;
    s.v = (float *)pk.v.p;
    s.f_nc = (float *)pk.fnc.p;
    s.f_cons = (float *)pk.fcons.p;
    s.masses = (const float *)pk.masses.p;
    s.energy = (double *)pk.energy.p;
    s.step = (uint64_t *)pk.step.p;
    s.seed = (const uint64_t *)pk.seed.p;
    s.replica_id = (const uint32_t *)pk.rid.p;
}

}  // namespace

extern "C" {

long long dmts_replica_footprint(const dmts_ctx *ctx, int n_atoms) {
    if (!ctx || n_atoms <= 0) return 0;
    // per-atom state (x, v, two force caches, x_ref, masses, species, mol, bonds)
    long long b = (long long)n_atoms * (4 * 12 + 12 + 4 + 1 + 4 + 4 * 4);
    // neighbour lists (about 80 + 40 entries per atom with head-room) and the
    // sorted rows kept between the count and the fill of a rebuild
    b += (long long)n_atoms * 4 * (160 + kNbrSlots);
    // activations of the conservative model
    const DevModel &m = ctx->cons;
    const int nlm = (m.lmax + 1) * (m.lmax + 1);
    b += (long long)n_atoms * m.C * 4 * (m.L + 1 + m.L * nlm + (m.lmax + 1) + m.L + 6 + nlm);
    // split-bf16 operand copies (hi and lo: 4 bytes per element) of q and of
    // the five [N][C] contraction inputs
    if (m.bf16) b += (long long)n_atoms * m.C * 4 * ((m.lmax + 1) + 5);
    return b;
}

dmts_status run_replicas(dmts_ctx *ctx, const dmts_request *reqs, int n_req, const dmts_integrator *p,
                         const dmts_serve_cfg *cfg, dmts_result *out, dmts_serve_stats *stats) {
    if (!ctx || (!reqs && n_req > 0) || !p || !cfg || (!out && n_req > 0) || n_req < 0)
        return fail(ctx, DMTS_E_INVALID, "run_replicas: NULL argument");
    if (!ctx->has_cons || (p->mode == DMTS_MODE_RESPA && !ctx->has_nc))
        return fail(ctx, DMTS_E_INVALID, "run_replicas: context lacks a model");
    if (cfg->max_slots < 1) return fail(ctx, DMTS_E_INVALID, "run_replicas: max_slots < 1");
    for (int k = 0; k < n_req; ++k) {
        const dmts_request &q = reqs[k];
        if (q.n_atoms < 1 || !q.x || !q.v || !q.species || !q.mol_id || !q.masses || q.n_outer < 0 ||
            (q.n_bonds > 0 && (!q.bonds || !q.bond_r0)))
            return fail(ctx, DMTS_E_INVALID, "run_replicas: malformed request");
        if (k > 0 && q.arrival_s < reqs[k - 1].arrival_s)
            return fail(ctx, DMTS_E_INVALID, "run_replicas: requests must be sorted by arrival time");
        if (!out[k].x || !out[k].v) return fail(ctx, DMTS_E_INVALID, "run_replicas: result buffers missing");
    }
    cudaSetDevice(ctx->device);
    cudaStream_t st = nullptr;
    if (!ck(ctx, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "run_replicas: stream")) return DMTS_E_CUDA;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    const int n_in = p->mode == DMTS_MODE_STS ? 1 : p->n_inner;

    Packed pk[2], adm;
    int cur = 0;
    dmts_state state, astate;
    memset(&state, 0, sizeof state);
    memset(&astate, 0, sizeof astate);
    Buf map;
    std::vector<Slot> slots;
    std::vector<int> waiting;
    long long footprint = 0;
    int next = 0, ticks_since_repack = kRepackTicks, n_ticks = 0, max_res = 0;
    double atom_steps = 0.0;
    dmts_status status = DMTS_OK;
    const auto t0 = std::chrono::steady_clock::now();
    for (int k = 0; k < n_req; ++k) {
        out[k].status = -1;
        out[k].t_arrival_s = reqs[k].arrival_s;
    }

    auto finish_copy = [&](Slot &sl, int off, int r) -> bool {
        const dmts_request &q = reqs[sl.req];
        dmts_result &o = out[sl.req];
        const bool ok =
            ck(ctx, cudaMemcpyAsync(o.x, (float *)pk[cur].x.p + 3 * off, sizeof(float) * 3 * q.n_atoms,
                                    cudaMemcpyDeviceToHost, st), "run_replicas: copy x") &&
            ck(ctx, cudaMemcpyAsync(o.v, (float *)pk[cur].v.p + 3 * off, sizeof(float) * 3 * q.n_atoms,
                                    cudaMemcpyDeviceToHost, st), "run_replicas: copy v") &&
            ck(ctx, cudaMemcpyAsync(&o.energy, (double *)pk[cur].energy.p + r, sizeof(double),
                                    cudaMemcpyDeviceToHost, st), "run_replicas: copy energy");
        sl.finished = true;
        o.t_done_s = now_s(t0);
        o.status = DMTS_OK;
        return ok;
    };

    while (status == DMTS_OK) {
        // ---- admission (arrival order, slots and memory permitting)
        const double tnow = now_s(t0);
        int live = 0;
        for (const Slot &sl : slots) live += !sl.finished;
        while (next < n_req && (!cfg->realtime || reqs[next].arrival_s <= tnow) &&
               live + (int)waiting.size() < cfg->max_slots) {
            const long long fp = dmts_replica_footprint(ctx, reqs[next].n_atoms);
            if (fp > cfg->hbm_budget_bytes) {
                out[next].status = DMTS_E_OOM;
                ++next;
                continue;
            }
            if (footprint + fp > cfg->hbm_budget_bytes) break;
            footprint += fp;
            waiting.push_back(next++);
        }
        // requests that need no steps finish at admission
        for (size_t w = 0; w < waiting.size();) {
            const dmts_request &q = reqs[waiting[w]];
            if (q.n_outer == 0) {
                memcpy(out[waiting[w]].x, q.x, sizeof(float) * 3 * q.n_atoms);
                memcpy(out[waiting[w]].v, q.v, sizeof(float) * 3 * q.n_atoms);
                out[waiting[w]].energy = 0.0;
                out[waiting[w]].t_admit_s = out[waiting[w]].t_done_s = now_s(t0);
                out[waiting[w]].status = DMTS_OK;
                footprint -= dmts_replica_footprint(ctx, q.n_atoms);
                waiting.erase(waiting.begin() + w);
            } else {
                ++w;
            }
        }
        bool any_finished = false;
        for (const Slot &sl : slots) any_finished |= sl.finished;
        const bool repack = (!waiting.empty() && (live == 0 || ticks_since_repack >= kRepackTicks)) ||
                            (any_finished && (live == 0 || ticks_since_repack >= kRepackTicks));
        if (repack) {
            // ---- first forces of the newcomers, in their own batch
            if (!waiting.empty()) {
                HostBatch ha;
                std::vector<uint64_t> z(waiting.size(), 0);
                if ((status = build_host_batch(reqs, waiting, z, ha)) != DMTS_OK) break;
                if (!upload_static(adm, ha, st)) { status = fail(ctx, DMTS_E_OOM, "run_replicas: admission buffers"); break; }
                size_t off = 0;
                for (int k : waiting) {
                    const dmts_request &q = reqs[k];
                    if (!ck(ctx, cudaMemcpyAsync((float *)adm.x.p + 3 * off, q.x, sizeof(float) * 3 * q.n_atoms,
                                                 cudaMemcpyHostToDevice, st), "run_replicas: upload x") ||
                        !ck(ctx, cudaMemcpyAsync((float *)adm.v.p + 3 * off, q.v, sizeof(float) * 3 * q.n_atoms,
                                                 cudaMemcpyHostToDevice, st), "run_replicas: upload v")) {
                        status = DMTS_E_CUDA;
                        break;
                    }
                    off += q.n_atoms;
                }
                if (status != DMTS_OK) break;
                fill_state(astate, adm, ha);
                astate.first_step = 1;
                if ((status = init_state(ctx, &astate, p->skin, st)) != DMTS_OK) break;
                if ((status = respa_step(ctx, &astate, p, 0, st)) != DMTS_OK) break;
            }
            // ---- new packed layout: continuing replicas, then newcomers
            std::vector<int> order;
            std::vector<uint64_t> steps;
            std::vector<Slot> nslots;
            std::vector<int> amap;
            int old_off = 0;
            for (const Slot &sl : slots) {
                if (!sl.finished) {
                    order.push_back(sl.req);
                    steps.push_back((uint64_t)sl.done * n_in);
                    nslots.push_back(sl);
                    for (int a = 0; a < sl.n; ++a) amap.push_back(old_off + a);
                } else {
                    footprint -= dmts_replica_footprint(ctx, sl.n);
                }
                old_off += sl.n;
            }
            const int n_keep_atoms = (int)amap.size();
            for (int k : waiting) {
                order.push_back(k);
                steps.push_back(0);
                nslots.push_back(Slot{k, reqs[k].n_atoms, 0, false});
                out[k].t_admit_s = now_s(t0);
                for (int a = 0; a < reqs[k].n_atoms; ++a) amap.push_back(-1);
            }
            const int nxt = 1 - cur;
            HostBatch hb;
            if ((status = build_host_batch(reqs, order, steps, hb)) != DMTS_OK) break;
            if (!upload_static(pk[nxt], hb, st)) { status = fail(ctx, DMTS_E_OOM, "run_replicas: batch buffers"); break; }
            const int N = hb.rep_off.back();
            if (n_keep_atoms > 0) {
                if (!map.ensure(sizeof(int) * (N + 1)) ||
                    !ck(ctx, cudaMemcpyAsync(map.p, amap.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st),
                        "run_replicas: map")) {
                    status = DMTS_E_OOM;
                    break;
                }
                k_gather_state<<<(N + 255) / 256, 256, 0, st>>>(
                    N, (const int *)map.p, (const float *)pk[cur].x.p, (const float *)pk[cur].v.p,
                    (const float *)pk[cur].fnc.p, (const float *)pk[cur].fcons.p, (float *)pk[nxt].x.p,
                    (float *)pk[nxt].v.p, (float *)pk[nxt].fnc.p, (float *)pk[nxt].fcons.p);
                count_launch();
            }
            if (!waiting.empty()) {
                const int na = astate.sys.n_atoms;
                const size_t o3 = 3 * (size_t)n_keep_atoms, b3 = sizeof(float) * 3 * na;
                bool ok = ck(ctx, cudaMemcpyAsync((float *)pk[nxt].x.p + o3, adm.x.p, b3, cudaMemcpyDeviceToDevice, st), "x") &&
                          ck(ctx, cudaMemcpyAsync((float *)pk[nxt].v.p + o3, adm.v.p, b3, cudaMemcpyDeviceToDevice, st), "v") &&
                          ck(ctx, cudaMemcpyAsync((float *)pk[nxt].fnc.p + o3, adm.fnc.p, b3, cudaMemcpyDeviceToDevice, st), "fnc") &&
                          ck(ctx, cudaMemcpyAsync((float *)pk[nxt].fcons.p + o3, adm.fcons.p, b3, cudaMemcpyDeviceToDevice, st), "fcons");
                if (!ok) { status = DMTS_E_CUDA; break; }
            }
            cur = nxt;
            slots.swap(nslots);
            waiting.clear();
            ticks_since_repack = 0;
            if (slots.empty()) {
                if (next >= n_req) break;
                continue;
            }
            fill_state(state, pk[cur], hb);
            state.first_step = 0;
            if ((status = init_state(ctx, &state, p->skin, st)) != DMTS_OK) break;
        }
        live = 0;
        for (const Slot &sl : slots) live += !sl.finished;
        if (live == 0) {
            if (next >= n_req && waiting.empty()) break;
            if (cfg->realtime && next < n_req) {
                const double wait = reqs[next].arrival_s - now_s(t0);
                if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
            }
            continue;
        }
        // ---- one batched outer step for every resident replica
        cudaEventRecord(ev0, st);
        if ((status = respa_run(ctx, &state, p, 1, st, nullptr)) != DMTS_OK) break;
        cudaEventRecord(ev1, st);
        if (!ck(ctx, cudaEventSynchronize(ev1), "run_replicas: tick")) { status = DMTS_E_CUDA; break; }
        int err = 0;
        cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (err) {
            cudaMemset(ctx->d_err, 0, sizeof(int));
            status = fail(ctx, (dmts_status)err, "run_replicas: device error during a tick");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        if (stats && stats->tick_ms && n_ticks < stats->tick_cap) stats->tick_ms[n_ticks] = ms;
        if (stats && stats->tick_atoms && n_ticks < stats->tick_cap) stats->tick_atoms[n_ticks] = state.sys.n_atoms;
        ++n_ticks;
        ++ticks_since_repack;
        int off = 0, r = 0, resident = 0;
        for (Slot &sl : slots) {
            if (!sl.finished) {
                sl.done += 1;
                atom_steps += sl.n;
                ++resident;
                if (sl.done >= reqs[sl.req].n_outer && !finish_copy(sl, off, r)) { status = DMTS_E_CUDA; break; }
            }
            off += sl.n;
            ++r;
        }
        max_res = std::max(max_res, resident);
        cudaStreamSynchronize(st);
    }
    cudaStreamSynchronize(st);
    if (stats) {
        stats->n_ticks = n_ticks;
        stats->wall_s = now_s(t0);
        stats->atom_outer_steps = atom_steps;
        stats->max_resident = max_res;
    }
    if (state.internal) free_state_internal((StateInternal *)state.internal);
    if (astate.internal) free_state_internal((StateInternal *)astate.internal);
    pk[0].release();
    pk[1].release();
    adm.release();
    map.release();
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaStreamDestroy(st);
    return status;
}

}  // extern "C"
