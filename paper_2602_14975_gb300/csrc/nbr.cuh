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
};

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
// Exclusive scan of n ints into out[n+1]; if capacity >= 0 and the total
// exceeds it, set the overflow error. total (nullable) receives the sum.
void scan_ints(const int *in, int n, int *out, long long capacity, long long *total, int *err,
               const int *gate, cudaStream_t st);

}  // namespace dmts
