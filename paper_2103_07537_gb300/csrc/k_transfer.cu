// Smoothed transfers (beyond the paper, whose prolongator is the tentative
// one): the field-block-diagonal prolongator
//   P_f = (I - W_f D_ff^{-1} A_ff) P^_f          for every field f,
// its explicit transpose R = P^T, the general Galerkin triple product
// A_c = R (A P) (Sec. 3) and the transfer kernels of the V-cycle.
//
// Storage of P and R: block CSR whose stored blocks hold only the F diagonal
// sub-blocks of fb x fb (field-major, row-major); the off-field sub-blocks
// are structurally zero because P never couples fields (eq. blocktransfers).
//
// Setup products are computed in FP64 with the multiplications and additions
// in a fixed order and without contraction (__dmul_rn / __dadd_rn), each
// output owned by one lane, so the hierarchy does not depend on scheduling.
#include <cuda_bf16.h>

#include "common.cuh"

namespace bamg {

// ---------------------------------------------------------------------------
// Symbolic phase of a row-wise sparse product, one warp per output row.  The
// distinct keys of the row go into a per-warp open-addressing hash table in
// shared memory (linear probing, atomicCAS insert), are compacted, ranked
// and written ascending to tmp_cols[row * cap ...]; count[row] = their number.
// Key sources:
//   yrp == nullptr: key = xmap ? xmap[xci[q]] : xci[q]         q in X row
//   yrp != nullptr: key = yci[k], k in Y row xci[q],            q in X row
// More than cap keys in a row sets kDevRowTooLong.
// ---------------------------------------------------------------------------
constexpr int kSymWarps = 4;
constexpr int kHashSlots = 1024;  // power of two, > 2 * (kSymCap + 32)
constexpr int kSymCap = 256;

__device__ __forceinline__ unsigned hash_slot(int key) {
    return ((unsigned)key * 2654435761u) & (kHashSlots - 1);
}

__global__ void __launch_bounds__(kSymWarps * 32)
    spgemm_symbolic_kernel(int nrows, const int* __restrict__ xrp, const int* __restrict__ xci,
                           const int* __restrict__ xmap, const int* __restrict__ yrp, const int* __restrict__ yci,
                           int* __restrict__ count, int* __restrict__ tmp_cols, int cap, int* err) {
    __shared__ int table[kSymWarps][kHashSlots];
    __shared__ int list[kSymWarps][kSymCap + 32];
    __shared__ int size[kSymWarps];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * kSymWarps + wid;
    if (row >= nrows) return;
    int* tab = table[wid];
    for (int t = lane; t < kHashSlots; t += 32) tab[t] = -1;
    if (lane == 0) size[wid] = 0;
    __syncwarp();
    bool overflow = false;
    // candidate stream: (q, k) pairs flattened 32 at a time
    const int q0 = xrp[row], q1 = xrp[row + 1];
    for (int q = q0; q < q1 && !overflow; q += (yrp ? 1 : 32)) {
        int k0 = 0, k1 = 1;
        if (yrp) {
            const int t = xci[q];
            k0 = yrp[t];
            k1 = yrp[t + 1];
        }
        for (int kb = k0; kb < k1 && !overflow; kb += 32) {
            int key = -1;
            if (yrp) {
                if (kb + lane < k1) key = yci[kb + lane];
            } else if (q + lane < q1) {
                const int t = xci[q + lane];
                key = xmap ? xmap[t] : t;
            }
            if (key >= 0) {
                unsigned slot = hash_slot(key);
                for (int probe = 0; probe < kHashSlots; ++probe) {
                    const int prev = atomicCAS(&tab[slot], -1, key);
                    if (prev == -1) {
                        atomicAdd(&size[wid], 1);
                        break;
                    }
                    if (prev == key) break;
                    slot = (slot + 1) & (kHashSlots - 1);
                }
            }
            __syncwarp();
            overflow = size[wid] > cap;  // at most 32 keys past cap: the table never fills
            __syncwarp();
        }
    }
    if (overflow) {
        if (lane == 0) {
            set_error(err, kDevRowTooLong);
            count[row] = 0;
        }
        return;
    }
    // compact the table into list (slot order), then rank the keys
    const int m = size[wid];
    int base = 0;
    for (int t0 = 0; t0 < kHashSlots; t0 += 32) {
        const int key = tab[t0 + lane];
        const unsigned full = __ballot_sync(0xffffffffu, key >= 0);
        if (key >= 0) list[wid][base + __popc(full & ((1u << lane) - 1u))] = key;
        base += __popc(full);
    }
    __syncwarp();
    for (int p = lane; p < m; p += 32) {
        const int key = list[wid][p];
        int rank = 0;
        for (int r = 0; r < m; ++r) rank += list[wid][r] < key;
        tmp_cols[(size_t)row * cap + rank] = key;
    }
    if (lane == 0) count[row] = m;
}

int spgemm_symbolic(int nrows, const int* xrp, const int* xci, const int* xmap, const int* yrp, const int* yci,
                    int* count, int* tmp_cols, int cap, int* err, cudaStream_t s) {
    if (nrows <= 0) return BAMG_OK;
    if (cap > kSymCap) return BAMG_EINVAL;
    spgemm_symbolic_kernel<<<ceil_div(nrows, kSymWarps), kSymWarps * 32, 0, s>>>(nrows, xrp, xci, xmap, yrp, yci,
                                                                                  count, tmp_cols, cap, err);
    return launched(1);
}

__device__ __forceinline__ int bsearch_col(const int* __restrict__ ci, int lo, int hi, int col) {
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (ci[m] < col) lo = m + 1;
        else hi = m;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// P values, one warp per fine row i; lane e <-> sub-block entry (f, r, c):
//   S_f[i,J][m][c] = sum over stored k of row i with agg(ci[k]) = J (stored
//                    order) of A[k][f*FB+m][f*FB+c]
//   P_f[i,J][r][c] = [J = agg(i), r = c] - w_{agg(i),f} sum_m Dinv_f,i[r][m] S[m][c]
// ---------------------------------------------------------------------------
template <int B, int FB>
__global__ void prolongator_numeric_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                           const double* __restrict__ vals, const double* __restrict__ dinv,
                                           const int* __restrict__ agg, const double* __restrict__ omega_p,
                                           const int* __restrict__ p_rp, const int* __restrict__ p_ci,
                                           double* __restrict__ p_v) {
    constexpr int F = B / FB, PB = F * FB * FB;
    const int i = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int k0 = rp[i], k1 = rp[i + 1];
    const int ai = agg[i];
    for (int e = lane; e < PB; e += 32) {
        const int f = e / (FB * FB), r = (e / FB) % FB, c = e % FB;
        const double* D = dinv + ((size_t)i * F + f) * FB * FB + (size_t)r * FB;
        const double w = omega_p[(size_t)ai * F + f];
        for (int q = p_rp[i]; q < p_rp[i + 1]; ++q) {
            const int J = p_ci[q];
            double S[FB];
#pragma unroll
            for (int m = 0; m < FB; ++m) S[m] = 0.0;
            for (int k = k0; k < k1; ++k) {
                if (agg[ci[k]] != J) continue;
                const double* blk = vals + (size_t)k * B * B + (size_t)(f * FB) * B + f * FB + c;
#pragma unroll
                for (int m = 0; m < FB; ++m) S[m] = __dadd_rn(S[m], blk[(size_t)m * B]);
            }
            double t = 0.0;
#pragma unroll
            for (int m = 0; m < FB; ++m) t = __dadd_rn(t, __dmul_rn(D[m], S[m]));
            const double delta = (J == ai && r == c) ? 1.0 : 0.0;
            p_v[(size_t)q * PB + e] = __dsub_rn(delta, __dmul_rn(w, t));
        }
    }
}

// R index lists: r_q[t] = position of coarse I in P's row r_i[t]
__global__ void transpose_index_kernel(int nc, const int* __restrict__ r_rp, const int* __restrict__ r_i,
                                       const int* __restrict__ p_rp, const int* __restrict__ p_ci,
                                       int* __restrict__ r_q, int* err) {
    const int I = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (I >= nc) return;
    for (int t = r_rp[I] + lane; t < r_rp[I + 1]; t += 32) {
        const int i = r_i[t];
        const int q = bsearch_col(p_ci, p_rp[i], p_rp[i + 1], I);
        if (q >= p_rp[i + 1] || p_ci[q] != I) {
            set_error(err, kDevBadPattern);
            r_q[t] = p_rp[i];
        } else {
            r_q[t] = q;
        }
    }
}

// (A P)[i, J]: warp per fine row, lane e <-> entry (r, c) of the b x b block:
// for stored k of row i (stored order), for stored q of P's row ci[k]
// (ascending J): out[J][r][c] += sum_s A[k][r][g*FB+s] P_g[q][s][c - g*FB], g = field of c
template <int B, int FB>
__global__ void ap_numeric_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                  const double* __restrict__ vals, const int* __restrict__ p_rp,
                                  const int* __restrict__ p_ci, const double* __restrict__ p_v,
                                  const int* __restrict__ ap_rp, const int* __restrict__ ap_ci,
                                  double* __restrict__ ap_v) {
    constexpr int F = B / FB, PB = F * FB * FB;
    const int i = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int a0 = ap_rp[i], a1 = ap_rp[i + 1];
    for (int e = lane; e < (a1 - a0) * B * B; e += 32) ap_v[(size_t)a0 * B * B + e] = 0.0;
    __syncwarp();
    for (int e = lane; e < B * B; e += 32) {
        const int r = e / B, c = e % B, g = c / FB, cl = c % FB;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            const double* A = vals + (size_t)k * B * B + (size_t)r * B + g * FB;
            for (int q = p_rp[j]; q < p_rp[j + 1]; ++q) {
                const int pos = bsearch_col(ap_ci, a0, a1, p_ci[q]);
                const double* P = p_v + (size_t)q * PB + (size_t)g * FB * FB + cl;
                double t = 0.0;
#pragma unroll
                for (int s2 = 0; s2 < FB; ++s2) t = __dadd_rn(t, __dmul_rn(A[s2], P[(size_t)s2 * FB]));
                double* o = ap_v + (size_t)pos * B * B + e;
                *o = __dadd_rn(*o, t);
            }
        }
    }
}

// A_c[I, J]: warp per coarse row, lane e <-> (r, c): for the fine i of R's
// row I (ascending), for stored a of (AP)'s row i (ascending J):
// out[J][r][c] += sum_u P_f[q][u][r - f*FB] (AP)[a][f*FB+u][c], f = field of r
template <int B, int FB>
__global__ void rap_general_numeric_kernel(int nc, const int* __restrict__ r_rp, const int* __restrict__ r_i,
                                           const int* __restrict__ r_q, const double* __restrict__ p_v,
                                           const int* __restrict__ ap_rp, const int* __restrict__ ap_ci,
                                           const double* __restrict__ ap_v, const int* __restrict__ rp_c,
                                           const int* __restrict__ ci_c, double* __restrict__ vals_c) {
    constexpr int F = B / FB, PB = F * FB * FB;
    const int I = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (I >= nc) return;
    const int c0 = rp_c[I], c1 = rp_c[I + 1];
    for (int e = lane; e < (c1 - c0) * B * B; e += 32) vals_c[(size_t)c0 * B * B + e] = 0.0;
    __syncwarp();
    for (int e = lane; e < B * B; e += 32) {
        const int r = e / B, c = e % B, f = r / FB, rl = r % FB;
        for (int t = r_rp[I]; t < r_rp[I + 1]; ++t) {
            const int i = r_i[t];
            const double* P = p_v + (size_t)r_q[t] * PB + (size_t)f * FB * FB + rl;
            for (int a = ap_rp[i]; a < ap_rp[i + 1]; ++a) {
                const int pos = bsearch_col(ci_c, c0, c1, ap_ci[a]);
                const double* X = ap_v + (size_t)a * B * B + (size_t)(f * FB) * B + c;
                double sum = 0.0;
#pragma unroll
                for (int u = 0; u < FB; ++u) sum = __dadd_rn(sum, __dmul_rn(P[(size_t)u * FB], X[(size_t)u * B]));
                double* o = vals_c + (size_t)pos * B * B + e;
                *o = __dadd_rn(*o, sum);
            }
        }
    }
}

#define BAMG_FDIAG_CASES(M) BAMG_BLOCK_SHAPES(M)

int prolongator_numeric(int b, int fb, int n, const int* rp, const int* ci, const double* vals, const double* dinv,
                        const int* agg, const double* omega_p, const int* p_rp, const int* p_ci, double* p_v,
                        cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    const int grid = ceil_div((long)n * 32, 128);
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                             \
    case BB * 16 + FF:                                                                                           \
        prolongator_numeric_kernel<BB, FF><<<grid, 128, 0, s>>>(n, rp, ci, vals, dinv, agg, omega_p, p_rp, p_ci, \
                                                                p_v);                                            \
        break;
        BAMG_FDIAG_CASES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}

int transpose_index(int nc, const int* r_rp, const int* r_i, const int* p_rp, const int* p_ci, int* r_q, int* err,
                    cudaStream_t s) {
    if (nc <= 0) return BAMG_OK;
    transpose_index_kernel<<<ceil_div((long)nc * 32, 128), 128, 0, s>>>(nc, r_rp, r_i, p_rp, p_ci, r_q, err);
    return launched(1);
}

int ap_numeric(int b, int fb, int n, const int* rp, const int* ci, const double* vals, const int* p_rp,
               const int* p_ci, const double* p_v, const int* ap_rp, const int* ap_ci, double* ap_v, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    const int grid = ceil_div((long)n * 32, 128);
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                          \
    case BB * 16 + FF:                                                                                        \
        ap_numeric_kernel<BB, FF><<<grid, 128, 0, s>>>(n, rp, ci, vals, p_rp, p_ci, p_v, ap_rp, ap_ci, ap_v); \
        break;
        BAMG_FDIAG_CASES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}

int rap_general_numeric(int b, int fb, int nc, const int* r_rp, const int* r_i, const int* r_q, const double* p_v,
                        const int* ap_rp, const int* ap_ci, const double* ap_v, const int* rp_c, const int* ci_c,
                        double* vals_c, cudaStream_t s) {
    if (nc <= 0) return BAMG_OK;
    const int grid = ceil_div((long)nc * 32, 128);
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                              \
    case BB * 16 + FF:                                                                                            \
        rap_general_numeric_kernel<BB, FF><<<grid, 128, 0, s>>>(nc, r_rp, r_i, r_q, p_v, ap_rp, ap_ci, ap_v, rp_c, \
                                                                ci_c, vals_c);                                    \
        break;
        BAMG_FDIAG_CASES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}

// ---------------------------------------------------------------------------
// values of P and R in the cycle's storage type V (FP64, FP32 or BF16):
// P copied, R[t] = the transposed sub-blocks of P[r_q[t]]
// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ V to_storage(double x);
template <>
__device__ __forceinline__ double to_storage<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_storage<float>(double x) { return (float)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16>(double x) {
    return __float2bfloat16_rn((float)x);
}

template <typename V>
__global__ void transfer_values_kernel(long nnz, int F, int fb, const int* __restrict__ r_q,
                                       const double* __restrict__ p_v, V* __restrict__ p_out, V* __restrict__ r_out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int PB = F * fb * fb;
    if (e >= nnz * PB) return;
    p_out[e] = to_storage<V>(p_v[e]);
    const long t = e / PB;
    const int w = (int)(e % PB);
    const int f = w / (fb * fb), rl = (w / fb) % fb, m = w % fb;
    // R_f[t][rl][m] = P_f[r_q[t]][m][rl]
    r_out[e] = to_storage<V>(p_v[(size_t)r_q[t] * PB + (size_t)f * fb * fb + (size_t)m * fb + rl]);
}

template <typename V>
int transfer_values(long nnz, int F, int fb, const int* r_q, const double* p_v, V* p_out, V* r_out, cudaStream_t s) {
    if (nnz <= 0) return BAMG_OK;
    transfer_values_kernel<V><<<ceil_div(nnz * F * fb * fb, 256), 256, 0, s>>>(nnz, F, fb, r_q, p_v, p_out, r_out);
    return launched(1);
}
template int transfer_values<double>(long, int, int, const int*, const double*, double*, double*, cudaStream_t);
template int transfer_values<float>(long, int, int, const int*, const double*, float*, float*, cudaStream_t);
template int transfer_values<__nv_bfloat16>(long, int, int, const int*, const double*, __nv_bfloat16*,
                                            __nv_bfloat16*, cudaStream_t);

// ---------------------------------------------------------------------------
// Transfers of the V-cycle with an explicit field-block-diagonal operator M
// (R for the restriction, P for the prolongation), one thread per output dof
// (row, d), f = d / FB, rl = d % FB:
//   y[row][d] (+)= sum over stored k of the row of sum_m M_f[k][rl][m] x[col_k][f*FB+m]
// Consecutive threads read consecutive sub-block rows of one stored block.
// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ float from_storage(V v);
template <>
__device__ __forceinline__ float from_storage<float>(float v) { return v; }
template <>
__device__ __forceinline__ float from_storage<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T, typename V, int B, int FB, bool ADD>
__global__ void __launch_bounds__(256) fdiag_spmv_kernel(int nrows, const int* __restrict__ rp,
                                                          const int* __restrict__ ci, const V* __restrict__ vals,
                                                          const T* __restrict__ x, T* __restrict__ y) {
    constexpr int F = B / FB, PB = F * FB * FB;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)nrows * B) return;
    const int row = (int)(e / B), d = (int)(e % B);
    const int f = d / FB, rl = d % FB;
    const int k0 = __ldg(rp + row), k1 = __ldg(rp + row + 1);
    pdl_wait();
    pdl_trigger();
    T acc = T(0);
    for (int k = k0; k < k1; ++k) {
        const int col = __ldg(ci + k);
        const V* m = vals + (size_t)k * PB + (size_t)f * FB * FB + (size_t)rl * FB;
        const T* xc = x + (size_t)col * B + f * FB;
#pragma unroll
        for (int u = 0; u < FB; ++u) {
            T mv;
            if constexpr (sizeof(V) == sizeof(T)) mv = m[u];
            else mv = (T)from_storage<V>(m[u]);
            acc = fma(mv, xc[u], acc);
        }
    }
    if (ADD) y[e] += acc;
    else y[e] = acc;
}

template <typename T, typename V>
int launch_fdiag_spmv(int b, int fb, int nrows, const int* rp, const int* ci, const V* vals, const T* x, T* y,
                      bool add, cudaStream_t s) {
    if (nrows <= 0) return BAMG_OK;
    const int grid = ceil_div((long)nrows * b, 256);
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                             \
    case BB * 16 + FF:                                                                                           \
        if ((add ? launch_k(fdiag_spmv_kernel<T, V, BB, FF, true>, grid, 256, 0, s, nrows, rp, ci, vals, x, y)     \
                 : launch_k(fdiag_spmv_kernel<T, V, BB, FF, false>, grid, 256, 0, s, nrows, rp, ci, vals, x, y)) != \
            cudaSuccess)                                                                                          \
            return BAMG_ECUDA;                                                                                    \
        break;
        BAMG_FDIAG_CASES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_fdiag_spmv<double, double>(int, int, int, const int*, const int*, const double*, const double*,
                                               double*, bool, cudaStream_t);
template int launch_fdiag_spmv<float, float>(int, int, int, const int*, const int*, const float*, const float*,
                                             float*, bool, cudaStream_t);
template int launch_fdiag_spmv<float, __nv_bfloat16>(int, int, int, const int*, const int*, const __nv_bfloat16*,
                                                     const float*, float*, bool, cudaStream_t);

}  // namespace bamg
