// Neighbour build for callers that cannot allocate device memory: the same
// cell-list kernels as nbr_build, with every scratch buffer carved out of one
// file-scope device array of fixed size.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "engine.cuh"

using namespace dmts;

namespace {

constexpr int kMaxAtoms = DMTS_STATIC_MAX_ATOMS;
constexpr int kMaxCells = DMTS_STATIC_MAX_CELLS;
constexpr int kMaxReplicas = DMTS_STATIC_MAX_REPLICAS;
constexpr int kMaxDevices = 64;

// Layout of the scratch array (byte offsets, each 256-aligned).
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffGrid = 0;
constexpr size_t kOffCellCnt = kOffGrid + align256(sizeof(CellGrid) * kMaxReplicas);
constexpr size_t kOffCellStart = kOffCellCnt + align256(sizeof(int) * kMaxCells);
constexpr size_t kOffCellAtoms = kOffCellStart + align256(sizeof(int) * (kMaxCells + 1));
constexpr size_t kOffAtomCell = kOffCellAtoms + align256(sizeof(int) * kMaxAtoms);
constexpr size_t kOffAtomSlot = kOffAtomCell + align256(sizeof(int) * kMaxAtoms);
constexpr size_t kOffCounts = kOffAtomSlot + align256(sizeof(int) * kMaxAtoms);
constexpr size_t kOffAtomRep = kOffCounts + align256(sizeof(int) * kMaxAtoms);
constexpr size_t kOffTotal = kOffAtomRep + align256(sizeof(int) * kMaxAtoms);
constexpr size_t kOffErr = kOffTotal + align256(sizeof(long long));
constexpr int kScanTiles = (std::max(kMaxAtoms, kMaxCells) + kScanTile - 1) / kScanTile + 1;
constexpr size_t kOffScan = kOffErr + align256(sizeof(int));   // prefix-scan status words and tile counters
constexpr size_t kScratchBytes = kOffScan + align256(sizeof(unsigned long long) * (2 * kScanTiles + 2));

}  // namespace

// Shared by every call on a device, kept until the process exits.
static __device__ __align__(256) unsigned char g_nbr_scratch[kScratchBytes];

static std::mutex g_setup_mutex;
static unsigned char *g_scratch_ptr[kMaxDevices];

// Device address of g_nbr_scratch on the current device, looked up once per
// device (the host-side name of the array is not a device address).
static dmts_status scratch_address(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(nullptr, DMTS_E_CUDA, "nbr_build_noalloc: no current CUDA device");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_nbr_scratch);
        if (e != cudaSuccess || !p) {
            ck(nullptr, e, "nbr_build_noalloc: cudaGetSymbolAddress");
            return DMTS_E_CUDA;
        }
        g_scratch_ptr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_ptr[dev];
    return DMTS_OK;
}

extern "C" dmts_status nbr_build_noalloc(const dmts_system *sys, dmts_nbr *nbr, long long *n_pairs,
                                         void *stream) {
    if (!sys || !nbr || !nbr->row_ptr || (!nbr->col && nbr->capacity > 0) || !(nbr->r_list > 0.f))
        return fail(nullptr, DMTS_E_INVALID, "nbr_build_noalloc: bad argument");
    if (sys->n_atoms < 0 || sys->n_replicas < 1 || !sys->rep_off || !sys->box || (sys->n_atoms > 0 && !sys->x))
        return fail(nullptr, DMTS_E_INVALID, "nbr_build_noalloc: bad system");
    if (sys->n_atoms > kMaxAtoms || sys->n_replicas > kMaxReplicas)
        return fail(nullptr, DMTS_E_INVALID,
                    "nbr_build_noalloc: more than DMTS_STATIC_MAX_ATOMS atoms or DMTS_STATIC_MAX_REPLICAS replicas");
    unsigned char *base = nullptr;
    dmts_status s = scratch_address(&base);
    if (s != DMTS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int R = sys->n_replicas, N = sys->n_atoms;

    // replica offsets and boxes on the host (fixed-size arrays, no heap)
    static thread_local int h_off[kMaxReplicas + 1];
    static thread_local float h_box[3 * kMaxReplicas];
    static thread_local CellGrid h_grid[kMaxReplicas];
    if (!ck(nullptr, cudaMemcpyAsync(h_off, sys->rep_off, sizeof(int) * (R + 1), cudaMemcpyDeviceToHost, st),
            "nbr_build_noalloc: rep_off") ||
        !ck(nullptr, cudaMemcpyAsync(h_box, sys->box, sizeof(float) * 3 * R, cudaMemcpyDeviceToHost, st),
            "nbr_build_noalloc: box") ||
        !ck(nullptr, cudaStreamSynchronize(st), "nbr_build_noalloc: synchronize"))
        return DMTS_E_CUDA;
    if (h_off[0] != 0 || h_off[R] != N) return fail(nullptr, DMTS_E_INVALID, "nbr_build_noalloc: rep_off inconsistent");
    int n_cells = 0;
    for (int r = 0; r < R; ++r) {
        CellGrid g;
        memset(&g, 0, sizeof g);
        const bool periodic = h_box[3 * r] > 0.f;
        for (int a = 0; a < 3; ++a) {
            const float L = h_box[3 * r + a];
            if (periodic != (L > 0.f))
                return fail(nullptr, DMTS_E_INVALID, "nbr_build_noalloc: box must be periodic on all axes or none");
            if (periodic) {
                if (!(nbr->r_list < 0.5f * L))
                    return fail(nullptr, DMTS_E_INVALID, "nbr_build_noalloc: list cutoff must be < box/2");
                g.box[a] = L;
                g.dim[a] = std::max(1, std::min(64, (int)std::floor(L / nbr->r_list)));
                g.inv_h[a] = (float)g.dim[a] / L;
            } else {
                const int nr = h_off[r + 1] - h_off[r];
                g.dim[a] = std::max(1, std::min(32, (int)std::lround(std::cbrt(nr / 8.0))));
                g.inv_h[a] = 1.f / nbr->r_list;
            }
        }
        g.cell_off = n_cells;
        n_cells += g.dim[0] * g.dim[1] * g.dim[2];
        if (n_cells > kMaxCells)
            return fail(nullptr, DMTS_E_INVALID, "nbr_build_noalloc: more than DMTS_STATIC_MAX_CELLS cells");
        h_grid[r] = g;
    }

    NbrWork w;
    w.n_atoms = N;
    w.n_rep = R;
    w.n_cells = n_cells;
    w.x = sys->x;
    w.rep_off = sys->rep_off;
    int *atom_rep = (int *)(base + kOffAtomRep);
    w.atom_rep = atom_rep;
    w.grid = (CellGrid *)(base + kOffGrid);
    w.cell_cnt = (int *)(base + kOffCellCnt);
    w.cell_start = (int *)(base + kOffCellStart);
    w.cell_atoms = (int *)(base + kOffCellAtoms);
    w.atom_cell = (int *)(base + kOffAtomCell);
    w.atom_slot = (int *)(base + kOffAtomSlot);
    w.counts = (int *)(base + kOffCounts);
    w.total = (long long *)(base + kOffTotal);
    w.gate = nullptr;
    w.err = (int *)(base + kOffErr);
    w.scan_status = (unsigned long long *)(base + kOffScan);
    w.scan_counter = w.scan_status + 2 * (size_t)kScanTiles;
    w.scan_tiles = kScanTiles;
    // the previous call's contents are still there: clear the words that
    // must start at zero (error word, total; nbr_cells clears the counts)
    if (!ck(nullptr, cudaMemsetAsync(base + kOffTotal, 0, kScratchBytes - kOffTotal, st), "nbr_build_noalloc: clear") ||
        !ck(nullptr, cudaMemcpyAsync(w.grid, h_grid, sizeof(CellGrid) * R, cudaMemcpyHostToDevice, st),
            "nbr_build_noalloc: grid"))
        return DMTS_E_CUDA;
    // an empty system launches nothing: its one row offset is written here
    if (N == 0 && !ck(nullptr, cudaMemsetAsync(nbr->row_ptr, 0, sizeof(int), st), "nbr_build_noalloc: row_ptr"))
        return DMTS_E_CUDA;
    atom_rep_map(sys->rep_off, R, N, atom_rep, st);
    nbr_cells(w, nbr->r_list, st);
    nbr_fill(w, nbr->r_list, nbr->row_ptr, nbr->col, nbr->capacity, nullptr, st);
    long long tot = 0;
    int err = 0;
    if (!ck(nullptr, cudaMemcpyAsync(&tot, w.total, sizeof(long long), cudaMemcpyDeviceToHost, st), "nbr_build_noalloc: count") ||
        !ck(nullptr, cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st), "nbr_build_noalloc: error word") ||
        !ck(nullptr, cudaStreamSynchronize(st), "nbr_build_noalloc"))
        return DMTS_E_CUDA;
    if (n_pairs) *n_pairs = tot;
    if (err == DMTS_E_NBR_OVERFLOW) return fail(nullptr, DMTS_E_NBR_OVERFLOW, "nbr_build_noalloc: capacity too small");
    if (err) return fail(nullptr, (dmts_status)err, "nbr_build_noalloc: device error");
    return DMTS_OK;
}
