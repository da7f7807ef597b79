// Solve-phase kernels of the V-cycle (Fig. 1 of the paper) and its building
// blocks: block-CSR SpMV / residual, restriction and prolongation with the
// piecewise-constant transfers of Sec. 4.3.1, one colour of the block
// Gauss-Seidel smoother of Algorithm 1 (Sec. 4.3.2), the dense coarsest
// solve, and precision casts at the cycle boundary.
//
// Thread mapping.  One warp per block row (node): its lanes cover (block,
// scalar row) pairs of the row, so one load instruction of a warp reads a
// contiguous run of the row's blocks, and values are loaded with the widest
// aligned vector type for the block size.  Short rows (9 blocks in 2D) are
// covered in one or two passes, which keeps the dependent-load chain of a
// warp short: these kernels are latency bound on L2-resident levels.
#include "common.cuh"

namespace bamg {

// ---------------------------------------------------------------------------
// Row reductions.  One warp owns one block row; lane = kk * R + r handles
// row r (r < R) of block kk + pass * G (G = 32 / R blocks per pass), so the
// lanes of a pass read consecutive rows of consecutive blocks (contiguous
// memory).  The partial sums of the lanes with the same r are then added by
// a shuffle tree whose offsets are multiples of R.
// ---------------------------------------------------------------------------
// largest R * 2^p below the warp size: the first offset of the shuffle tree
template <int R>
struct RowTree {
    static constexpr int kStart = (R * 16 < kWarp) ? R * 16 : (R * 8 < kWarp) ? R * 8 : (R * 4 < kWarp) ? R * 4
                                  : (R * 2 < kWarp) ? R * 2 : R;
};

template <typename T, int R>
__device__ __forceinline__ T reduce_rows(T v, int lane) {
#pragma unroll
    for (int off = RowTree<R>::kStart; off >= R; off >>= 1) {
        const T o = __shfl_down_sync(0xffffffffu, v, off);
        if (lane + off < kWarp) v += o;
    }
    return v;  // lanes 0..R-1 hold the row sums
}

// ---------------------------------------------------------------------------
// y = A x, or y = rhs - A x: one warp per block row
// ---------------------------------------------------------------------------
template <typename T, int B>
__global__ void __launch_bounds__(256) spmv_kernel(int n, const int* __restrict__ rp,
                                                   const int* __restrict__ ci,
                                                   const T* __restrict__ vals, const T* __restrict__ x,
                                                   const T* __restrict__ rhs, T* __restrict__ y) {
    constexpr int G = kWarp / B;
    const long i = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;  // uniform per warp
    const int lane = threadIdx.x & (kWarp - 1);
    const int kk = lane / B;
    const int r = lane - kk * B;
    const int k0 = __ldg(rp + i), k1 = __ldg(rp + i + 1);
    T acc = T(0);
    if (kk < G) {
        for (int k = k0 + kk; k < k1; k += G) {
            const int j = __ldg(ci + k);
            T a[B], xv[B];
            load_row<T, B>(vals + (size_t)k * B * B + r * B, a);
            load_row<T, B>(x + (size_t)j * B, xv);
#pragma unroll
            for (int c = 0; c < B; ++c) acc = fma(a[c], xv[c], acc);
        }
    }
    acc = reduce_rows<T, B>(acc, lane);
    if (lane < B) y[(size_t)i * B + lane] = rhs ? rhs[(size_t)i * B + lane] - acc : acc;
}

template <typename T>
int launch_spmv(int b, int n, const int* rp, const int* ci, const T* vals, const T* x, const T* rhs,
                T* y, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    const int threads = 256;
    const int blocks = ceil_div((long)n * kWarp, threads);
    switch (b) {
#define CASE(BB) \
    case BB: spmv_kernel<T, BB><<<blocks, threads, 0, s>>>(n, rp, ci, vals, x, rhs, y); break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_spmv<double>(int, int, const int*, const int*, const double*, const double*,
                                 const double*, double*, cudaStream_t);
template int launch_spmv<float>(int, int, const int*, const int*, const float*, const float*,
                                const float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// restriction with R = P^T, P piecewise constant: rc[I,d] = sum_{m in I} res[m,d]
// members ascending, so the sum order is fixed (deterministic).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void restrict_kernel(int b, int nc, const int* __restrict__ agg_ptr,
                                const int* __restrict__ members, const T* __restrict__ res,
                                T* __restrict__ rc) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int I = (int)(t / b);
    const int d = (int)(t - (long)I * b);
    if (I >= nc) return;
    T acc = T(0);
    for (int q = agg_ptr[I]; q < agg_ptr[I + 1]; ++q) acc += res[(size_t)members[q] * b + d];
    rc[(size_t)I * b + d] = acc;
}

template <typename T>
int launch_restrict(int b, int nc, const int* agg_ptr, const int* members, const T* res, T* rc,
                    cudaStream_t s) {
    if (nc <= 0) return BAMG_OK;
    restrict_kernel<T><<<ceil_div((long)nc * b, 256), 256, 0, s>>>(b, nc, agg_ptr, members, res, rc);
    return launched(1);
}
template int launch_restrict<double>(int, int, const int*, const int*, const double*, double*, cudaStream_t);
template int launch_restrict<float>(int, int, const int*, const int*, const float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// prolongation and correction u += P uc, P piecewise constant per dof
// ---------------------------------------------------------------------------
template <typename T>
__global__ void prolong_kernel(int b, int n, const int* __restrict__ agg, const T* __restrict__ uc,
                               T* __restrict__ u) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(e / b);
    if (i >= n) return;
    const int d = (int)(e - (long)i * b);
    u[e] += uc[(size_t)agg[i] * b + d];
}

template <typename T>
int launch_prolong(int b, int n, const int* agg, const T* uc, T* u, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    prolong_kernel<T><<<ceil_div((long)n * b, 256), 256, 0, s>>>(b, n, agg, uc, u);
    return launched(1);
}
template int launch_prolong<double>(int, int, const int*, const double*, double*, cudaStream_t);
template int launch_prolong<float>(int, int, const int*, const float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// One colour of one field step of the damped block Gauss-Seidel smoother
// (Algorithm 1).  For field f the step computes
//   r_f = rhs_f - A_{f,*} x                 (x = x_in, fixed for the whole step)
//   x~  = one multicolour node-block GS sweep on A_ff r_f from x~ = 0:
//         x~_i = D_ff,i^{-1} (r_f,i - sum_{j != i} A_ff[i,j] x~_j)
//   x_f = x_f + omega x~_f
// The residual and the Gauss-Seidel sum read the same f-rows of each block,
// so they are fused into one pass: node i of colour c accumulates
//   rhs_f,i - sum_j A_{f,*}[i,j] x_in,j - sum_{j: colour(j) < c} A_ff[i,j] x~_j
// (neighbours of later colours still have x~ = 0, neighbours of the same
// colour do not exist).  x_in is never written during the step; node i writes
// its updated values to x_out (all b components: field f corrected, the
// others copied), so the fields' update of Algorithm 1 needs no extra pass.
// The fb threads of node i sit in one warp and exchange their row sums by
// shuffles for the fb x fb inverse.
// ---------------------------------------------------------------------------
template <typename T, int B, int FB>
__global__ void __launch_bounds__(256) bgs_colour_kernel(BgsArgs a) {
    constexpr int G = kWarp / FB;  // blocks of the row per pass
    const long q = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= a.n_in_colour) return;  // uniform per warp
    const int lane = threadIdx.x & (kWarp - 1);
    const int kk = lane / FB;
    const int r = lane - kk * FB;
    const int f0 = a.field * FB;
    const T* __restrict__ vals = static_cast<const T*>(a.vals);
    const T* __restrict__ x_in = static_cast<const T*>(a.x_in);
    const T* __restrict__ uc = static_cast<const T*>(a.uc);
    const T* __restrict__ xt = static_cast<const T*>(a.xt);
    const int i = __ldg(a.nodes + q);
    const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1);
    // the fb x fb inverse row of this lane (lanes r < FB), loaded early
    T drow[FB];
    if (lane < FB) {
        const T* D = static_cast<const T*>(a.dinv) + ((size_t)i * a.F + a.field) * FB * FB + (size_t)lane * FB;
#pragma unroll
        for (int c = 0; c < FB; ++c) drow[c] = D[c];
    }
    T acc = T(0);
    if (kk < G) {
        for (int k = k0 + kk; k < k1; k += G) {
            const int j = __ldg(a.ci + k);
            T arow[B];
            load_row<T, B>(vals + (size_t)k * B * B + (size_t)(f0 + r) * B, arow);
            if (x_in) {
                T xv[B];
                load_row<T, B>(x_in + (size_t)j * B, xv);
                if (uc) {  // prolongation fused in: x = x_in + P uc
                    T pv[B];
                    load_row<T, B>(uc + (size_t)__ldg(a.agg + j) * B, pv);
#pragma unroll
                    for (int c = 0; c < B; ++c) xv[c] += pv[c];
                }
#pragma unroll
                for (int c = 0; c < B; ++c) acc = fma(arow[c], xv[c], acc);
            }
            if (j != i && __ldg(a.colours + j) < a.colour) {
                const T* tv = xt + (size_t)j * FB;
                // field-f columns of the row with compile-time register indices
#pragma unroll
                for (int ff = 0; ff < B / FB; ++ff)
                    if (ff == a.field) {
#pragma unroll
                        for (int c = 0; c < FB; ++c) acc = fma(arow[ff * FB + c], tv[c], acc);
                    }
            }
        }
    }
    acc = reduce_rows<T, FB>(acc, lane);
    // lanes 0..FB-1: the row sums of A_{f,*} x + A_ff x~ for this node
    T t = T(0);
    if (lane < FB) t = static_cast<const T*>(a.rhs)[(size_t)i * B + f0 + lane] - acc;
    T xn = T(0);
#pragma unroll
    for (int c = 0; c < FB; ++c) {
        const T tc = __shfl_sync(0xffffffffu, t, c);
        if (lane < FB) xn = fma(drow[c], tc, xn);
    }
    if (lane < FB) static_cast<T*>(a.xt)[(size_t)i * FB + lane] = xn;
    // x_out for node i: every component copied (with the prolongation when
    // fused), field f corrected by omega x~
    const T xf = __shfl_sync(0xffffffffu, xn, (lane - f0) & (kWarp - 1));
    if (lane < B) {
        const size_t e = (size_t)i * B + lane;
        T v = x_in ? x_in[e] : T(0);
        if (x_in && uc) v += uc[(size_t)__ldg(a.agg + i) * B + lane];
        if (lane >= f0 && lane < f0 + FB) v = fma(T(a.omega), xf, v);
        static_cast<T*>(a.x_out)[e] = v;
    }
}

template <typename T>
int launch_bgs_colour(int b, int fb, const BgsArgs& a, cudaStream_t s) {
    if (a.n_in_colour <= 0) return BAMG_OK;
    const int threads = 256;
    const int blocks = ceil_div((long)a.n_in_colour * kWarp, threads);
    switch (b * 16 + fb) {
#define CASE(BB, FF) \
    case BB * 16 + FF: bgs_colour_kernel<T, BB, FF><<<blocks, threads, 0, s>>>(a); break;
        CASE(1, 1) CASE(2, 2) CASE(3, 3) CASE(4, 4) CASE(4, 2) CASE(6, 6) CASE(6, 3)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_bgs_colour<double>(int, int, const BgsArgs&, cudaStream_t);
template int launch_bgs_colour<float>(int, int, const BgsArgs&, cudaStream_t);

// ---------------------------------------------------------------------------
// coarsest level: y = A_L^{-1} x with the FP64 inverse, one warp per row
// ---------------------------------------------------------------------------
template <typename T>
__global__ void dense_gemv_kernel(int nd, const double* __restrict__ ainv, const T* __restrict__ x,
                                  T* __restrict__ y) {
    const int row = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= nd) return;
    const double* a = ainv + (size_t)row * nd;
    double acc = 0.0;
    for (int c = lane; c < nd; c += kWarp) acc = fma(a[c], (double)x[c], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[row] = (T)acc;
}

template <typename T>
int launch_dense_gemv(int nd, const double* ainv, const T* x, T* y, cudaStream_t s) {
    if (nd <= 0) return BAMG_OK;
    dense_gemv_kernel<T><<<ceil_div((long)nd * kWarp, 256), 256, 0, s>>>(nd, ainv, x, y);
    return launched(1);
}
template int launch_dense_gemv<double>(int, const double*, const double*, double*, cudaStream_t);
template int launch_dense_gemv<float>(int, const double*, const float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// precision casts at the cycle boundary (FP64 Krylov vectors <-> FP32 cycle)
// ---------------------------------------------------------------------------
__global__ void cast_d2f_kernel(long m, const double* __restrict__ x, float* __restrict__ y) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (long)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
}
__global__ void cast_f2d_kernel(long m, const float* __restrict__ x, double* __restrict__ y) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (long)gridDim.x * blockDim.x)
        y[e] = (double)x[e];
}
static int grid_for(long m) {
    long g = (m + 255) / 256;
    return (int)(g < 152L * 16 ? (g > 0 ? g : 1) : 152L * 16);
}
int launch_cast_d2f(long m, const double* x, float* y, cudaStream_t s) {
    if (m <= 0) return BAMG_OK;
    cast_d2f_kernel<<<grid_for(m), 256, 0, s>>>(m, x, y);
    return launched(1);
}
int launch_cast_f2d(long m, const float* x, double* y, cudaStream_t s) {
    if (m <= 0) return BAMG_OK;
    cast_f2d_kernel<<<grid_for(m), 256, 0, s>>>(m, x, y);
    return launched(1);
}

}  // namespace bamg
