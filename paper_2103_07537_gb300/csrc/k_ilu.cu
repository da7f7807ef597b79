// ILU(0) of each field's diagonal part as the sub-solve of Algorithm 1
// (Sec. 4.3.2: the paper approximates every A_ff^{-1} by an incomplete
// factorisation; Sec. 5.1), in the multicolour elimination order.
//
// A_ff is the scalar matrix of the fb x fb field-f sub-blocks of the stored
// blocks.  The nodes are eliminated colour by colour (colour, then index: the
// level's colour-ordered node list), scalar rows of a node in dof order.  The
// nodes of one colour do not couple, so each colour's nodes are factored in
// parallel (one thread per node, the node's rows in order), and each colour's
// rows of the forward (colours ascending) and backward (colours descending)
// triangular solves are independent: one launch per colour and direction, as
// the multicolour Gauss-Seidel sweep has one per colour.
//
// Factor layout: lu[f][k][r][c] (one plane of nnzb fb x fb sub-blocks per
// field).  Entry (k, r, c) of block k = (i, j) holds L (unit lower, strictly
// before the scalar diagonal in elimination order) or U (on and after it).
// The factorisation repeats the operations of the definition in its order
// (rows ascending; for each entry q < p of row p, l = a_pq / u_qq, then
// a_pt -= l u_qt for every t > q held by rows p and q), in FP64 without
// contraction, so its factors are those of a sequential elimination.
#include "common.cuh"
#include "bgs_body.cuh"

namespace bamg {

// lu[f][k] = the field-f sub-block of block k (all fields)
__global__ void ilu_copy_kernel(long nnzb, int b, int fb, int F, const double* __restrict__ vals,
                                double* __restrict__ lu) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long ff = (long)fb * fb;
    if (t >= (long)F * nnzb * ff) return;
    const int f = (int)(t / (nnzb * ff));
    const long rem = t - (long)f * nnzb * ff;
    const long k = rem / ff;
    const int rc = (int)(rem - k * ff), r = rc / fb, c = rc - r * fb;
    lu[t] = vals[k * b * b + (long)(f * fb + r) * b + f * fb + c];
}

// position of every node in the colour-ordered node list
__global__ void ilu_pos_kernel(int n, const int* __restrict__ nodes, int* __restrict__ pos) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) pos[nodes[p]] = p;
}

// upk[k] = 1 where block k of row i has a column j of higher colour (and, with
// node fields, of the same field): the U part a backward solve reads
__global__ void ilu_upper_flags_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                       const int* __restrict__ colour, const int* __restrict__ node_field,
                                       unsigned char* __restrict__ upk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        upk[k] = (j != i && colour[j] > colour[i] && (!node_field || node_field[j] == node_field[i])) ? 1 : 0;
    }
}

constexpr int kIluMaxRow = 64;  // stored blocks per row the factorisation takes

__device__ __forceinline__ int find_block(const int* __restrict__ ci, int k0, int k1, int col) {
    while (k0 < k1) {
        const int m = (k0 + k1) >> 1;
        const int v = ci[m];
        if (v == col) return m;
        if (v < col) k0 = m + 1;
        else k1 = m;
    }
    return -1;
}

// one colour's nodes of one field plane, a thread per node
__global__ void ilu_factor_colour_kernel(int n_in_colour, const int* __restrict__ nodes, const int* __restrict__ rp,
                                         const int* __restrict__ ci, const int* __restrict__ pos,
                                         const int* __restrict__ diag, const int* __restrict__ node_field, int fb,
                                         double* __restrict__ lu, int* err) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_in_colour) return;
    const int i = nodes[q];
    const int e = pos[i];
    const int k0 = rp[i], k1 = rp[i + 1];
    const int gi = node_field ? node_field[i] : 0;
    const size_t ff = (size_t)fb * fb;
    // the row's blocks (of the node's field) by elimination position of the column
    int order[kIluMaxRow];
    int len = 0;
    for (int k = k0; k < k1; ++k) {
        if (node_field && node_field[ci[k]] != gi) continue;
        if (len == kIluMaxRow) {
            set_error(err, kDevRowTooLong);
            return;
        }
        int u = len++;
        const int ek = pos[ci[k]];
        while (u > 0 && pos[ci[order[u - 1]]] > ek) {
            order[u] = order[u - 1];
            --u;
        }
        order[u] = k;
    }
    for (int r = 0; r < fb; ++r) {
        const int p = e * fb + r;
        for (int t = 0; t < len; ++t) {
            const int k = order[t];
            const int j = ci[k];
            const int e2 = pos[j];
            if (e2 > e) break;
            const int kd = diag[j];
            for (int c = 0; c < fb; ++c) {
                const int qq = e2 * fb + c;
                if (qq >= p) continue;
                const double uqq = lu[(size_t)kd * ff + c * fb + c];
                if (uqq == 0.0) {
                    set_error(err, kDevSingularBlock);
                    return;
                }
                const double l = __ddiv_rn(lu[(size_t)k * ff + r * fb + c], uqq);
                lu[(size_t)k * ff + r * fb + c] = l;
                // a_pt -= l u_qt for t > q held by both rows (row i in stored order)
                for (int k2 = k0; k2 < k1; ++k2) {
                    const int j2 = ci[k2];
                    if (node_field && node_field[j2] != gi) continue;
                    const int kq = find_block(ci, rp[j], rp[j + 1], j2);
                    if (kq < 0) continue;
                    const int e3 = pos[j2];
                    for (int c2 = 0; c2 < fb; ++c2) {
                        if (e3 * fb + c2 <= qq) continue;
                        double* a = lu + (size_t)k2 * ff + r * fb + c2;
                        *a = __dsub_rn(*a, __dmul_rn(l, lu[(size_t)kq * ff + c * fb + c2]));
                    }
                }
            }
        }
    }
    // the pivots of the node's own rows
    const int kd = diag[i];
    for (int r = 0; r < fb; ++r)
        if (lu[(size_t)kd * ff + r * fb + r] == 0.0) set_error(err, kDevSingularBlock);
}

int ilu_factor(int n, int b, int fb, int F, long nnzb, int n_colours, const std::vector<int>& colour_ptr,
               const int* nodes, const int* rp, const int* ci, const int* diag, const int* node_field,
               const double* vals, int* pos, double* lu, int* err, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    const long tot = (long)F * nnzb * fb * fb;
    ilu_copy_kernel<<<ceil_div(tot, 256), 256, 0, s>>>(nnzb, b, fb, F, vals, lu);
    ilu_pos_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, nodes, pos);
    int launches = 2;
    for (int f = 0; f < F; ++f)
        for (int c = 0; c < n_colours; ++c) {
            const int m = colour_ptr[c + 1] - colour_ptr[c];
            if (m <= 0) continue;
            ilu_factor_colour_kernel<<<ceil_div(m, 128), 128, 0, s>>>(m, nodes + colour_ptr[c], rp, ci, pos, diag,
                                                                     node_field, fb, lu + (size_t)f * nnzb * fb * fb,
                                                                     err);
            ++launches;
        }
    return launched(launches);
}

int launch_upper_flags(int n, const int* rp, const int* ci, const int* colour, const int* node_field,
                       unsigned char* upk, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    ilu_upper_flags_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, ci, colour, node_field, upk);
    return launched(1);
}

// ---------------------------------------------------------------------------
// triangular solves of one field step, one colour per launch, one thread per
// scalar row (FB threads per node; the node's own fb x fb triangle is solved
// by the node's first thread after the off-node sums)
// ---------------------------------------------------------------------------
template <int FB>
struct IluBlock {
    static constexpr int kThreads = RowThreads<FB>::kThreads;
};

// forward: y_i = L_ii^{-1} (r_f,i - sum_{lower j} L_ij y_j), where the field's
// residual r_f = rhs_f - A_{f,*} x_in is formed in the same pass (x_in + P uc
// when uc is set); y goes to xt
template <typename T, int B, int FB, bool FM>
__global__ void __launch_bounds__(IluBlock<FB>::kThreads) ilu_fwd_kernel(BgsArgs a, const T* __restrict__ lu,
                                                                         const int* __restrict__ diag) {
    constexpr int NT = IluBlock<FB>::kThreads;
    __shared__ T sh[NT];
    const int nloc = threadIdx.x / FB, r = threadIdx.x - nloc * FB;
    const long q = (long)blockIdx.x * (NT / FB) + nloc;
    const bool act = q < a.n_in_colour;
    const int f0 = a.field * FB;
    const T* __restrict__ vals = static_cast<const T*>(a.vals);
    const T* __restrict__ x_in = static_cast<const T*>(a.x_in);
    const T* __restrict__ uc = static_cast<const T*>(a.uc);
    T* xt = static_cast<T*>(a.xt);
    pdl_wait();
    pdl_trigger();
    int i = 0;
    T acc = T(0);
    if (act) {
        i = __ldg(a.nodes + q);
        const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1);
        const T* vb = vrow<T, B, FB, FM>(vals, k0, k1, k0, f0 + r);
        constexpr int VS = vstride<T, B, FB, FM>();
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const bool lower = __ldg(a.lowk + k) != 0;
            if (!x_in && !lower) continue;
            const int j = __ldg(a.ci + k);
            if (x_in) {
                T arow[B], xv[B];
                load_row<T, B>(vb + (size_t)(k - k0) * VS, arow);
                load_row<T, B>(x_in + (size_t)j * B, xv);
                if (uc) {
                    T pv[B];
                    load_row<T, B>(uc + (size_t)__ldg(a.agg + j) * B, pv);
#pragma unroll
                    for (int c = 0; c < B; ++c) xv[c] += pv[c];
                }
#pragma unroll
                for (int c = 0; c < B; ++c) acc = fma(arow[c], xv[c], acc);
            }
            if (lower) {
                T lrow[FB], yv[FB];
                load_row<T, FB>(lu + (size_t)k * FB * FB + r * FB, lrow);
                load_row<T, FB>(xt + (size_t)j * FB, yv);
#pragma unroll
                for (int c = 0; c < FB; ++c) acc = fma(lrow[c], yv[c], acc);
            }
        }
        sh[nloc * FB + r] = static_cast<const T*>(a.rhs)[(size_t)i * B + f0 + r] - acc;
    }
    __syncthreads();
    if (act && r == 0) {
        const T* Ld = lu + (size_t)__ldg(diag + i) * FB * FB;
        T y[FB];
#pragma unroll
        for (int rr = 0; rr < FB; ++rr) {
            T s = sh[nloc * FB + rr];
#pragma unroll
            for (int c = 0; c < rr; ++c) s -= Ld[rr * FB + c] * y[c];
            y[rr] = s;
        }
#pragma unroll
        for (int rr = 0; rr < FB; ++rr) xt[(size_t)i * FB + rr] = y[rr];
    }
}

// backward: x~_i = U_ii^{-1} (y_i - sum_{higher j} U_ij x~_j) in place of y in
// xt, then x_out = x_in (+ P uc) with field f += omega x~
template <typename T, int B, int FB>
__global__ void __launch_bounds__(IluBlock<FB>::kThreads) ilu_bwd_kernel(BgsArgs a, const T* __restrict__ lu,
                                                                         const int* __restrict__ diag,
                                                                         const unsigned char* __restrict__ upk) {
    constexpr int NT = IluBlock<FB>::kThreads;
    __shared__ T sh[NT];
    const int nloc = threadIdx.x / FB, r = threadIdx.x - nloc * FB;
    const long q = (long)blockIdx.x * (NT / FB) + nloc;
    const bool act = q < a.n_in_colour;
    const T* __restrict__ x_in = static_cast<const T*>(a.x_in);
    const T* __restrict__ uc = static_cast<const T*>(a.uc);
    T* xt = static_cast<T*>(a.xt);
    pdl_wait();
    pdl_trigger();
    int i = 0;
    if (act) {
        i = __ldg(a.nodes + q);
        const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1);
        T acc = T(0);
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            if (!__ldg(upk + k)) continue;
            const int j = __ldg(a.ci + k);
            T urow[FB], xv[FB];
            load_row<T, FB>(lu + (size_t)k * FB * FB + r * FB, urow);
            load_row<T, FB>(xt + (size_t)j * FB, xv);
#pragma unroll
            for (int c = 0; c < FB; ++c) acc = fma(urow[c], xv[c], acc);
        }
        sh[nloc * FB + r] = xt[(size_t)i * FB + r] - acc;
    }
    __syncthreads();
    if (act && r == 0) {
        const T* Ud = lu + (size_t)__ldg(diag + i) * FB * FB;
        T x[FB];
#pragma unroll
        for (int rr = FB - 1; rr >= 0; --rr) {
            T s = sh[nloc * FB + rr];
#pragma unroll
            for (int c = rr + 1; c < FB; ++c) s -= Ud[rr * FB + c] * x[c];
            x[rr] = s / Ud[rr * FB + rr];
        }
#pragma unroll
        for (int rr = 0; rr < FB; ++rr) sh[nloc * FB + rr] = x[rr];
    }
    __syncthreads();
    if (!act) return;
    const T xn = sh[nloc * FB + r];
    xt[(size_t)i * FB + r] = xn;
    T* __restrict__ x_out = static_cast<T*>(a.x_out);
    const T om = a.omega_node ? static_cast<const T*>(a.omega_node)[(size_t)i * a.F + a.field] : T(a.omega);
    const int ag = (x_in && uc) ? __ldg(a.agg + i) : 0;
    for (int m = 0; m < a.F; ++m) {
        const size_t e = (size_t)i * B + m * FB + r;
        T v = x_in ? x_in[e] : T(0);
        if (x_in && uc) v += uc[(size_t)ag * B + m * FB + r];
        if (m == a.field) v = fma(om, xn, v);
        x_out[e] = v;
    }
}

template <typename T>
int launch_ilu_colour(int b, int fb, const BgsArgs& a, const T* lu, const int* diag, const unsigned char* upk,
                      bool backward, cudaStream_t s) {
    if (a.n_in_colour <= 0) return BAMG_OK;
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                          \
    case BB * 16 + FF: {                                                                                      \
        constexpr int NT = IluBlock<FF>::kThreads;                                                            \
        constexpr bool kFm = HasFm<T, BB, FF>::value;                                                        \
        const int grid = ceil_div(a.n_in_colour, NT / FF);                                                   \
        cudaError_t e;                                                                                        \
        if (backward) e = launch_k(ilu_bwd_kernel<T, BB, FF>, grid, NT, 0, s, a, lu, diag, upk);             \
        else if (a.fm && kFm) e = launch_k(ilu_fwd_kernel<T, BB, FF, kFm>, grid, NT, 0, s, a, lu, diag);     \
        else e = launch_k(ilu_fwd_kernel<T, BB, FF, false>, grid, NT, 0, s, a, lu, diag);                    \
        if (e != cudaSuccess) return BAMG_ECUDA;                                                              \
        break;                                                                                                \
    }
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_ilu_colour<double>(int, int, const BgsArgs&, const double*, const int*, const unsigned char*,
                                       bool, cudaStream_t);
template int launch_ilu_colour<float>(int, int, const BgsArgs&, const float*, const int*, const unsigned char*, bool,
                                      cudaStream_t);

}  // namespace bamg
