// Per-kernel CUDA-event timing (instrumentation of the measurement harness).
#include <atomic>
#include <cstring>
#include <string>

#include "engine.cuh"

namespace dmts {

static std::atomic<unsigned long long> g_kernel_launches{0};

void count_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(unsigned long long n) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_kernel_launches.load(std::memory_order_relaxed); }

int Profiler::slot(const char *name) {
    for (size_t k = 0; k < slots.size(); ++k)
        if (slots[k].name == name) return (int)k;
    slots.push_back(ProfSlot{name, {}, 0, 0.0});
    return (int)slots.size() - 1;
}

cudaEvent_t Profiler::take() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void Profiler::flush() {
    for (auto &s : slots) {
        for (auto &pr : s.ev) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) s.ms += ms;
            pool.push_back(pr.first);
            pool.push_back(pr.second);
        }
        s.ev.clear();
    }
}

void Profiler::clear() {
    flush();
    slots.clear();
}

void Profiler::release() {
    clear();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
}

ProfScope::ProfScope(dmts_ctx *ctx, const char *name, cudaStream_t st) : p(nullptr), s(st), k(-1) {
    if (!ctx || !ctx->prof.on || !ctx->prof.active) return;
    p = &ctx->prof;
    k = p->slot(name);
    start = p->take();
    cudaEventRecord(start, st);
}

ProfScope::~ProfScope() {
    if (!p) return;
    cudaEvent_t stop = p->take();
    cudaEventRecord(stop, s);
    p->slots[k].ev.emplace_back(start, stop);
    p->slots[k].launches++;
    if (p->slots[k].ev.size() > 4096) {   // bound the number of pending events
        cudaEventSynchronize(stop);
        p->flush();
    }
}

}  // namespace dmts

using namespace dmts;

extern "C" {

dmts_status dmts_profile_enable(dmts_ctx *ctx, int enable) {
    if (!ctx) return DMTS_E_INVALID;
    cudaSetDevice(ctx->device);
    if (enable) {
        cudaDeviceSynchronize();
        ctx->prof.clear();
    }
    ctx->prof.on = enable != 0;
    ctx->prof.every = enable > 1 ? enable : 1;
    ctx->prof.outer = 0;
    ctx->prof.active = true;
    return DMTS_OK;
}

int dmts_profile_read(dmts_ctx *ctx, int idx, char *name, int name_cap, long long *launches, double *total_ms) {
    if (!ctx) return -1;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    ctx->prof.flush();
    if (idx < 0) return (int)ctx->prof.slots.size();
    if (idx >= (int)ctx->prof.slots.size()) return -1;
    const ProfSlot &s = ctx->prof.slots[idx];
    if (name && name_cap > 0) {
        strncpy(name, s.name.c_str(), name_cap - 1);
        name[name_cap - 1] = 0;
    }
    if (launches) *launches = s.launches;
    if (total_ms) *total_ms = s.ms;
    return 0;
}

unsigned long long dmts_kernel_launches(void) { return dmts::g_kernel_launches.load(std::memory_order_relaxed); }

}  // extern "C"
