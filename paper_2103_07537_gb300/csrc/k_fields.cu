// Setup kernels for fields on disjoint node sets: the graph of the diagonal
// field blocks (the input of the separate aggregation and colouring of every
// field, Sec. 4.3.1), per-field colour ranges and the field-restricted
// lower-colour flags of Algorithm 1's sub-solve.  One thread per node; every
// index read comes from a pattern that the level's pattern check accepted
// (columns in range) or from node_field (values 0..nf-1 by construction).
#include "common.cuh"
#include "fields.cuh"

namespace bamg {

__global__ void field_count_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                   const int* __restrict__ node_field, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int f = node_field[i];
    int c = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) c += node_field[ci[k]] == f;
    count[i] = c;
}

__global__ void field_fill_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                  const int* __restrict__ node_field, const int* __restrict__ rp_f,
                                  int* __restrict__ ci_f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int f = node_field[i];
    int e = rp_f[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        if (node_field[j] == f) ci_f[e++] = j;
    }
}

int field_pattern(int n, const int* rp, const int* ci, const int* node_field, int* count, int* scan_tmp,
                  long scan_bytes, int* rp_f, int* ci_f, cudaStream_t s) {
    if (n <= 0) return BAMG_EINVAL;
    field_count_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, ci, node_field, count);
    note_launch(1);
    int st = exclusive_scan(n, count, rp_f, scan_tmp, scan_bytes, s);
    if (st) return st;
    field_fill_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, ci, node_field, rp_f, ci_f);
    return launched(1);
}

__global__ void field_colour_max_kernel(int n, const int* __restrict__ colour, const int* __restrict__ node_field,
                                        int* __restrict__ cmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(cmax + node_field[i], colour[i] + 1);
}

int field_colour_counts(int n, int nf, const int* colour, const int* node_field, int* cmax, cudaStream_t s) {
    if (n <= 0 || nf <= 0) return BAMG_EINVAL;
    BAMG_CUDA_TRY(cudaMemsetAsync(cmax, 0, sizeof(int) * (size_t)nf, s));
    field_colour_max_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, colour, node_field, cmax);
    return launched(1);
}

__global__ void field_colour_shift_kernel(int n, const int* __restrict__ colour_off,
                                          const int* __restrict__ node_field, int* __restrict__ colour) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) colour[i] += colour_off[node_field[i]];
}

int field_colour_shift(int n, const int* colour_off, const int* node_field, int* colour, cudaStream_t s) {
    if (n <= 0) return BAMG_EINVAL;
    field_colour_shift_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, colour_off, node_field, colour);
    return launched(1);
}

__global__ void field_lower_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                   const int* __restrict__ colour, const int* __restrict__ node_field,
                                   unsigned char* __restrict__ lowk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = colour[i], f = node_field[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        lowk[k] = (j != i && node_field[j] == f && colour[j] < c) ? 1 : 0;
    }
}

int field_lower_flags(int n, const int* rp, const int* ci, const int* colour, const int* node_field,
                      unsigned char* lowk, cudaStream_t s) {
    if (n <= 0) return BAMG_EINVAL;
    field_lower_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, ci, colour, node_field, lowk);
    return launched(1);
}

}  // namespace bamg
