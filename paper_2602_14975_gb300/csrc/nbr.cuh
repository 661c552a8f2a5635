// Cell-list neighbour build: a full list and, in the same pass, the sub-list
// of its entries within a shorter cutoff.
#pragma once
#include "common.cuh"

namespace dmts {

// Cell grid of one replica. Periodic replicas: origin 0, edge box/dim.
// Open replicas: origin and edge set on the device from the bounding box.
struct CellGrid {
    float org[3];
    float inv_h[3];
    float box[3];       // 0 on an open axis
    int dim[3];
    int cell_off;       // first global cell index of this replica
};

struct NbrWork {
    // sizes
    int n_atoms, n_rep, n_cells;
    // inputs
    const float *x;
    const int *rep_off;
    const int *atom_rep;
    CellGrid *grid;       // [n_rep] (device)
    // scratch
    int *cell_cnt;        // [n_cells]
    int *cell_start;      // [n_cells+1]
    int *cell_atoms;      // [n_atoms]
    int *atom_cell;       // [n_atoms]
    int *atom_slot;       // [n_atoms]
    int *counts;          // [n_atoms]
    long long *total;     // [1] device: pairs needed by the last fill
    const int *gate;      // nullable: skip everything when *gate == 0
    int *err;             // sticky error word
    int *counts_sub = nullptr;   // [n_atoms]: row lengths of the sub-list (nbr_fill with a sub-list)
    int *slots = nullptr;        // [n_atoms][slot_cap] (nullable): sorted rows kept by the count pass
    int slot_cap = 0;
    const float *box = nullptr;  // [n_rep][3] (nullable): current boxes; periodic grids follow them at each
                                 // rebuild (a barostat moves the box)
    // prefix-scan state: per job [scan_tiles] tile status words and a word
    // holding the scan's epoch (upper 32 bits) and the tiles taken so far
    // (lower 32, zero between scans); the epoch tags the status words, so a
    // scan never reads an earlier scan's words and no launch argument
    // changes from one scan to the next (graph replays)
    unsigned long long *scan_status = nullptr;   // [2][scan_tiles]
    unsigned long long *scan_counter = nullptr;  // [2]
    int scan_tiles = 0;
};

// Tiles of the prefix scan (elements per tile) and the tiles a scan of n
// elements needs.
constexpr int kScanTile = 2048;
inline int scan_tiles_for(int n) { return (n + kScanTile - 1) / kScanTile + 1; }

// Builds the cell structure (assign, count, scan, scatter, sort).
void nbr_cells(const NbrWork &w, float r_list, cudaStream_t st);
// Count + scan + fill of a full list within r_list using the cell structure.
// x_ref (nullable) receives the positions used. With sub_col (and
// w.counts_sub) the same pass also writes the sub-list of entries within
// r_sub < r_list (rows in the same ascending order).
void nbr_fill(const NbrWork &w, float r_list, int *row_ptr, int *col, long long capacity,
              float *x_ref, cudaStream_t st, float r_sub = 0.f, int *sub_row = nullptr, int *sub_col = nullptr,
              long long sub_capacity = -1);
// Atom -> replica map.
void atom_rep_map(const int *rep_off, int n_rep, int n_atoms, int *atom_rep, cudaStream_t st);
// Exclusive scans of n ints into out[n+1], one or two arrays in one launch
// (in1 nullable); if capacity >= 0 and a total exceeds it, set the overflow
// error; total (nullable) receives the sum. Single pass over the whole grid:
// tiles of kScanTile elements publish their sums and look back at their
// predecessors' (decoupled look-back), every wait bounded.
void scan_ints(const NbrWork &w, const int *in0, int *out0, long long cap0, long long *total0, const int *in1,
               int *out1, long long cap1, long long *total1, int n, cudaStream_t st);

}  // namespace dmts
