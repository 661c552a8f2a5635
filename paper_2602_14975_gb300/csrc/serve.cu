// Continuous-batching serving loop over independent replicas.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "engine.cuh"

using namespace dmts;

extern "C" {

long long dmts_replica_footprint(const dmts_ctx *ctx, int n_atoms) {
    if (!ctx || n_atoms <= 0) return 0;
    // per-atom state (x, v, two force caches, x_ref, masses, species, mol, bonds)
    long long b = (long long)n_atoms * (4 * 12 + 12 + 4 + 1 + 4 + 4 * 4);
    // neighbour lists (about 80 + 40 entries per atom with head-room)
    b += (long long)n_atoms * 4 * 160;
    // activations of the conservative model
    const DevModel &m = ctx->cons;
    const int nlm = (m.lmax + 1) * (m.lmax + 1);
    b += (long long)n_atoms * m.C * 4 * (m.L + 1 + m.L * nlm + (m.lmax + 1) + m.L + 6 + nlm);
    return b;
}

dmts_status run_replicas(dmts_ctx *ctx, const dmts_request *reqs, int n_req, const dmts_integrator *p,
                         const dmts_serve_cfg *cfg, dmts_result *out, dmts_serve_stats *stats) {
    (void)reqs; (void)n_req; (void)p; (void)cfg; (void)out; (void)stats;
    return fail(ctx, DMTS_E_INVALID, "run_replicas: serving loop not built yet");
}

}  // extern "C"
