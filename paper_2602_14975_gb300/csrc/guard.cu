// Rewind procedure around Algorithm 1 (Sec. 2, "Preventing rare model
// disagreements (Rewind procedure)"): saved frames every chunk, a per-replica
// monitor of |F - F_S| filled by the integrator's outer kicks, and on a
// disagreement (or a non-finite value) a return to the last frame followed by
// single-time-step BAOAB before Algorithm 1 resumes.
#include <cmath>
#include <cstring>
#include <vector>

#include "engine.cuh"

using namespace dmts;

namespace {

struct Frame {
    Buf x, v, f_nc, f_cons, step, energy, box, baro;
    int first_step = 0;

    bool alloc(int n, int n_rep, bool with_energy, bool with_baro) {
        return x.ensure(sizeof(float) * 3 * (size_t)(n + 1)) && v.ensure(sizeof(float) * 3 * (size_t)(n + 1)) &&
               f_nc.ensure(sizeof(float) * 3 * (size_t)(n + 1)) && f_cons.ensure(sizeof(float) * 3 * (size_t)(n + 1)) &&
               step.ensure(sizeof(uint64_t) * n_rep) && (!with_energy || energy.ensure(sizeof(double) * n_rep)) &&
               (!with_baro || (box.ensure(sizeof(float) * 3 * n_rep) && baro.ensure(sizeof(double) * 3 * n_rep)));
    }
    void release() {
        Buf *all[] = {&x, &v, &f_nc, &f_cons, &step, &energy, &box, &baro};
        for (Buf *b : all) b->release();
    }
};

// With the barostat the frame also holds the boxes and the piston state.
bool copy_state(dmts_ctx *ctx, Frame &f, dmts_state *s, bool save, cudaStream_t st) {
    const size_t b3 = sizeof(float) * 3 * (size_t)s->sys.n_atoms;
    const size_t br = (size_t)s->sys.n_replicas;
    struct Pair { void *frame; void *state; size_t bytes; } pairs[] = {
        {f.x.p, s->sys.x, b3}, {f.v.p, s->v, b3}, {f.f_nc.p, s->f_nc, b3}, {f.f_cons.p, s->f_cons, b3},
        {f.step.p, s->step, sizeof(uint64_t) * br}, {f.energy.p, s->energy, sizeof(double) * br},
        {f.box.p, const_cast<float *>(s->sys.box), sizeof(float) * 3 * br}, {f.baro.p, s->baro, sizeof(double) * 3 * br}};
    for (const Pair &pr : pairs) {
        if (!pr.frame || !pr.state || pr.bytes == 0) continue;
        const cudaError_t e = save ? cudaMemcpyAsync(pr.frame, pr.state, pr.bytes, cudaMemcpyDeviceToDevice, st)
                                   : cudaMemcpyAsync(pr.state, pr.frame, pr.bytes, cudaMemcpyDeviceToDevice, st);
        if (!ck(ctx, e, "saved frame copy")) return false;
    }
    if (save) f.first_step = s->first_step;
    else s->first_step = f.first_step;
    return true;
}

// Stream sync + error word: DMTS_OK, DMTS_E_NONFINITE (cleared, recoverable)
// or another device/CUDA error (returned as the call's status).
dmts_status settle(dmts_ctx *ctx, cudaStream_t st) {
    if (!ck(ctx, cudaStreamSynchronize(st), "stream synchronize")) return DMTS_E_CUDA;
    int err = 0;
    if (!ck(ctx, cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word")) return DMTS_E_CUDA;
    if (err) cudaMemset(ctx->d_err, 0, sizeof(int));
    return (dmts_status)err;
}

}  // namespace

extern "C" dmts_status respa_guarded(dmts_ctx *ctx, dmts_state *stt, const dmts_integrator *p,
                                     const dmts_guard *guard, int n_outer, dmts_guard_stats *stats, void *stream) {
    if (!ctx || !stt || !p || !guard) return fail(ctx, DMTS_E_INVALID, "NULL argument");
    if (p->mode != DMTS_MODE_RESPA) return fail(ctx, DMTS_E_INVALID, "the guard wraps Algorithm 1 (RESPA mode)");
    if (guard->chunk_outer < 1 || guard->sts_steps < 1 || !(guard->sts_dt > 0.f) || !(guard->threshold >= 0.f) ||
        n_outer < 0 || !(p->dt_outer > 0.f))
        return fail(ctx, DMTS_E_INVALID, "bad guard parameters");
    const double seg = (double)guard->sts_steps * guard->sts_dt / p->dt_outer;
    const int m_seg = (int)std::lround(seg);
    if (m_seg < 1 || std::fabs(seg - m_seg) > 1e-4) return fail(ctx, DMTS_E_INVALID, "sts_steps * sts_dt must be whole outer steps");
    if (!stt->f_nc || !stt->f_cons || !stt->v || !stt->step) return fail(ctx, DMTS_E_INVALID, "missing state array");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = stt->sys.n_atoms, R = stt->sys.n_replicas;
    if (stats) {
        stats->n_rewinds = 0;
        stats->n_chunks = 0;
    }
    Frame frame;
    Buf mon;
    const bool npt = p->barostat != 0;
    if (!frame.alloc(n, R, stt->energy != nullptr, npt) || !mon.ensure(sizeof(unsigned) * R)) {
        frame.release();
        return fail(ctx, DMTS_E_OOM, "saved frame allocation failed");
    }
    dmts_integrator ps = *p;
    ps.mode = DMTS_MODE_STS;
    ps.dt_outer = guard->sts_dt;
    ps.n_inner = 1;
    uint32_t thr_bits;
    std::memcpy(&thr_bits, &guard->threshold, sizeof thr_bits);
    std::vector<unsigned> host(R);
    dmts_status s = DMTS_OK;
    int done = 0;
    if (!copy_state(ctx, frame, stt, true, st)) s = DMTS_E_CUDA;
    while (s == DMTS_OK && done < n_outer) {
        const int c = std::min(guard->chunk_outer, n_outer - done);
        if (!ck(ctx, cudaMemsetAsync(mon.p, 0, sizeof(unsigned) * R, st), "monitor reset")) { s = DMTS_E_CUDA; break; }
        s = respa_run(ctx, stt, p, c, st, (unsigned *)mon.p);
        if (s != DMTS_OK) break;
        if (!ck(ctx, cudaMemcpyAsync(host.data(), mon.p, sizeof(unsigned) * R, cudaMemcpyDeviceToHost, st),
                "monitor read")) { s = DMTS_E_CUDA; break; }
        dmts_status e = settle(ctx, st);
        if (e != DMTS_OK && e != DMTS_E_NONFINITE) { s = fail(ctx, e, "device error"); break; }
        unsigned top = 0;
        for (unsigned b : host) top = std::max(top, b);
        if (stats) {
            if (stats->chunk_max && stats->n_chunks < stats->chunk_cap) {
                float f;
                std::memcpy(&f, &top, sizeof f);
                stats->chunk_max[stats->n_chunks] = f;
            }
            stats->n_chunks++;
        }
        const bool disagree = e == DMTS_E_NONFINITE || top > thr_bits;
        if (!disagree) {
            done += c;
            if (!copy_state(ctx, frame, stt, true, st)) s = DMTS_E_CUDA;
            continue;
        }
        // rewind: back to the saved frame, single time steps, fresh caches
        if (stats) {
            if (stats->rewind_at && stats->n_rewinds < stats->rewind_cap) stats->rewind_at[stats->n_rewinds] = (float)done;
            stats->n_rewinds++;
        }
        if (!copy_state(ctx, frame, stt, false, st)) { s = DMTS_E_CUDA; break; }
        state_force_rebuild(ctx, stt, st);
        s = respa_run(ctx, stt, &ps, guard->sts_steps, st, nullptr);
        if (s != DMTS_OK) break;
        e = settle(ctx, st);
        if (e == DMTS_E_NONFINITE) { s = fail(ctx, e, "non-finite values in the single-time-step segment"); break; }
        if (e != DMTS_OK) { s = fail(ctx, e, "device error"); break; }
        stt->first_step = 1;     // the fast-force cache is stale after STS
        // the single-time-step segment keeps the box; the piston's force is
        // re-derived from the full force's virial at the next outer step
        if (npt && !ck(ctx, cudaMemset2DAsync(stt->baro + 2, 3 * sizeof(double), 0, sizeof(double), R, st),
                       "piston reset")) { s = DMTS_E_CUDA; break; }
        done += m_seg;
        if (!copy_state(ctx, frame, stt, true, st)) s = DMTS_E_CUDA;
    }
    cudaStreamSynchronize(st);
    frame.release();
    mon.release();
    return s;
}
