// Setup kernels for fields on disjoint node sets (fields that are not
// co-located; separate aggregation per field block, Sec. 4.3.1, and the
// mixed-element example of Sec. 5).  Field g owns the contiguous node range
// [off[g], off[g+1]); node_field[i] is the field of node i.
#pragma once

#include <cuda_runtime.h>

namespace bamg {

// The graph of the diagonal field blocks: the stored blocks (i, j) of a level
// with node_field[i] == node_field[j], in their stored (ascending) order.
// count: n + 1 ints of scratch; scan_tmp / scan_bytes: scratch of
// exclusive_scan for n.  rp_f (n + 1) is filled; ci_f must hold at least as
// many ints as the level has stored blocks.
int field_pattern(int n, const int* rp, const int* ci, const int* node_field, int* count, int* scan_tmp,
                  long scan_bytes, int* rp_f, int* ci_f, cudaStream_t s);

// cmax[g] = 1 + the largest colour of a node of field g (cmax: nf ints,
// zeroed here)
int field_colour_counts(int n, int nf, const int* colour, const int* node_field, int* cmax, cudaStream_t s);

// colour[i] += coff[node_field[i]]: the colours of field g follow those of
// fields 0..g-1
int field_colour_shift(int n, const int* colour_off, const int* node_field, int* colour, cudaStream_t s);

// lowk[k] = 1 for a stored block (i, j), j != i, of the same field with
// colour[j] < colour[i] (the blocks a field step reads x~ through)
int field_lower_flags(int n, const int* rp, const int* ci, const int* colour, const int* node_field,
                      unsigned char* lowk, cudaStream_t s);

}  // namespace bamg
