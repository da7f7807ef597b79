// Solve-phase kernels of the V-cycle (Fig. 1 of the paper) and its building
// blocks: block-CSR SpMV / residual, restriction and prolongation with the
// piecewise-constant transfers of Sec. 4.3.1, one colour of the block
// Gauss-Seidel smoother of Algorithm 1 (Sec. 4.3.2), the dense coarsest
// solve, precision casts at the cycle boundary, and the cluster "tail"
// kernel that runs every step of the cycle below a given level in one launch.
//
// Thread mapping.  One warp per block row (node): its lanes cover (block,
// scalar row) pairs of the row, so one load instruction of a warp reads a
// contiguous run of the row's blocks, and values are loaded with the widest
// aligned vector type for the block size.  Short rows (9 blocks in 2D) are
// covered in one or two passes, which keeps the dependent-load chain of a
// warp short: these kernels are latency bound on L2-resident levels.
//
// The warp-level bodies are device functions shared by the one-step kernels
// and the tail kernel.  Their template flag CG selects L2-coherent loads
// (ld.global.cg) for vectors that the same launch writes (the tail kernel);
// matrix data is read through the read-only path in both.
#include <cooperative_groups.h>

#include "bgs_body.cuh"
#include "common.cuh"

namespace cg = cooperative_groups;

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

// y_i = (rhs_i -) sum_j A_ij x_j for block row i; whole warp.  With PDL the
// lane's first block (column and matrix row, fixed for the cycle) is loaded
// before the wait on the previous kernel.
template <typename T, int B, int FB, bool CG, bool PDL = false, bool FM = false>
__device__ __forceinline__ void spmv_row(long i, int lane, const int* __restrict__ rp, const int* __restrict__ ci,
                                         const T* __restrict__ vals, const T* x, const T* rhs, T* y) {
    constexpr int G = kWarp / B;
    const int kk = lane / B;
    const int r = lane - kk * B;
    const int k0 = __ldg(rp + i), k1 = __ldg(rp + i + 1);
    const int kf = k0 + kk;
    const bool have = kk < G && kf < k1;
    int jf = 0;
    T af[B];
    if (have) {
        jf = __ldg(ci + kf);
        load_row<T, B>(vrow<T, B, FB, FM>(vals, k0, k1, kf, r), af);
    }
    if constexpr (PDL) {
        pdl_wait();
        pdl_trigger();
    }
    const T bi = (rhs && lane < B) ? ld1<T, CG>(rhs + (size_t)i * B + lane) : T(0);  // issued early
    T acc = T(0);
    if (have) {
        {
            T xv[B];
            load_vec<T, B, CG>(x + (size_t)jf * B, xv);
#pragma unroll
            for (int c = 0; c < B; ++c) acc = fma(af[c], xv[c], acc);
        }
#pragma unroll 4
        for (int k = kf + G; k < k1; k += G) {
            const int j = __ldg(ci + k);
            T a[B], xv[B];
            load_row<T, B>(vrow<T, B, FB, FM>(vals, k0, k1, k, r), a);
            load_vec<T, B, CG>(x + (size_t)j * B, xv);
#pragma unroll
            for (int c = 0; c < B; ++c) acc = fma(a[c], xv[c], acc);
        }
    }
    acc = reduce_rows<T, B>(acc, lane);
    if (lane < B) y[(size_t)i * B + lane] = rhs ? bi - acc : acc;
}

// ---------------------------------------------------------------------------
// One colour of one field step of the damped block Gauss-Seidel smoother
// (Algorithm 1), one node per warp.  For field f the step computes
//   r_f = rhs_f - A_{f,*} x                 (x = x_in, fixed for the whole step)
//   x~  = one multicolour node-block GS sweep on A_ff r_f from x~ = 0:
//         x~_i = D_ff,i^{-1} (r_f,i - sum_{j != i} A_ff[i,j] x~_j)
//   x_f = x_f + omega x~_f      (omega_i,f of node i when omega_node is set)
// The residual and the Gauss-Seidel sum read the same f-rows of each block,
// so they are fused into one pass: node i of colour c accumulates
//   rhs_f,i - sum_j A_{f,*}[i,j] x_in,j - sum_{j: colour(j) < c} A_ff[i,j] x~_j
// (neighbours of later colours still have x~ = 0, neighbours of the same
// colour do not exist).  x_in is never written during the step; node i writes
// its updated values to x_out (all b components: field f corrected, the
// others copied), so the field update of Algorithm 1 needs no extra pass.
// With uc set, x_in + P uc (the coarse correction) is read in place of x_in.
// ---------------------------------------------------------------------------
template <typename T, int B, int FB, bool CG, bool PDL = false, bool FM = false>
__device__ __forceinline__ void bgs_node(const BgsArgs& a, long q, int lane) {
    constexpr int G = kWarp / FB;  // blocks of the row per pass
    const int kk = lane / FB;
    const int r = lane - kk * FB;
    const int f0 = a.field * FB;
    const T* __restrict__ vals = static_cast<const T*>(a.vals);
    const T* x_in = static_cast<const T*>(a.x_in);
    const T* uc = static_cast<const T*>(a.uc);
    const T* xt = static_cast<const T*>(a.xt);
    const int i = __ldg(a.nodes + q);
    const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1);
    // the fb x fb inverse row of this lane (lanes r < FB), loaded early
    T drow[FB];
    if (lane < FB) {
        const T* D = static_cast<const T*>(a.dinv) + ((size_t)i * a.F + a.field) * FB * FB + (size_t)lane * FB;
#pragma unroll
        for (int c = 0; c < FB; ++c) drow[c] = __ldg(D + c);
    }
    // the lane's first block: its column, matrix row, colour test and
    // aggregate are fixed for the whole cycle, so they are loaded before the
    // wait on the previous kernel (with programmatic dependent launch they
    // overlap its tail)
    // (rows hold at least their diagonal block: the clamped index stays in
    // the row, and lanes without a first block load but never use it)
    const int kf = k0 + kk;
    const bool have = kk < G && kf < k1;
    const int kq = min(kf, k1 - 1);
    const int jf = __ldg(a.ci + kq);
    const bool lowf = __ldg(a.lowk + kq) != 0;
    // this lane's matrix row in the row's first block; block k's is vstride apart
    const T* vb = vrow<T, B, FB, FM>(vals, k0, k1, k0, f0 + r);
    constexpr int VS = vstride<T, B, FB, FM>();
    // from a zero iterate only blocks of lower colour contribute: the others'
    // matrix rows are not loaded
    T arf[B];
    if (x_in || lowf) load_row<T, B>(vb + (size_t)(kq - k0) * VS, arf);
    const int agf = (x_in && uc) ? __ldg(a.agg + jf) : 0;
    if constexpr (PDL) {  // everything below may depend on earlier kernels
        pdl_wait();
        pdl_trigger();
    }
    const T bi = lane < FB ? ld1<T, CG>(static_cast<const T*>(a.rhs) + (size_t)i * B + f0 + lane) : T(0);
    T acc = T(0);
    if (have) bgs_walk<T, B, FB, CG, G>(a, xt, x_in, uc, vb, VS, k0, kf, k1, jf, lowf, agf, arf, acc);
    acc = reduce_rows<T, FB>(acc, lane);
    // lanes 0..FB-1: the row sums of A_{f,*} x + A_ff x~ for this node
    T t = T(0);
    if (lane < FB) t = bi - acc;
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
        T v = x_in ? ld1<T, CG>(x_in + e) : T(0);
        if (x_in && uc) v += ld1<T, CG>(uc + (size_t)__ldg(a.agg + i) * B + lane);
        if (lane >= f0 && lane < f0 + FB) {
            const T om = a.omega_node ? static_cast<const T*>(a.omega_node)[(size_t)i * a.F + a.field] : T(a.omega);
            v = fma(om, xf, v);
        }
        static_cast<T*>(a.x_out)[e] = v;
    }
}

// coarsest level: y_row = sum_c Ainv[row][c] x_c, summed in the inverse's
// type S; whole warp
template <typename T, typename S, bool CG>
__device__ __forceinline__ void gemv_row(int row, int lane, int nd, const S* __restrict__ ainv, const T* x,
                                         T* y) {
    const S* a = ainv + (size_t)row * nd;
    // four accumulators (columns lane + 32 (4 t + u)): four independent
    // load pairs in flight per lane, summed in a fixed order
    S acc[4] = {S(0), S(0), S(0), S(0)};
    int c = lane;
    for (; c + 3 * kWarp < nd; c += 4 * kWarp) {
        S av[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            av[u] = __ldg(a + c + u * kWarp);
            xv[u] = (S)ld1<T, CG>(x + c + u * kWarp);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(av[u], xv[u], acc[u]);
    }
    for (int u = 0; c < nd; c += kWarp, ++u) acc[u] = fma(__ldg(a + c), (S)ld1<T, CG>(x + c), acc[u]);
    S sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    sum = warp_sum(sum);
    if (lane == 0) y[row] = (T)sum;
}

// restriction with R = P^T, P piecewise constant: rc[I,d] = sum_{m in I} res[m,d],
// members ascending, so the sum order is fixed (deterministic)
template <typename T, bool CG>
__device__ __forceinline__ void restrict_dof(long t, int b, const int* __restrict__ agg_ptr,
                                             const int* __restrict__ members, const T* res, T* rc) {
    const int I = (int)(t / b);
    const int d = (int)(t - (long)I * b);
    const int q0 = __ldg(agg_ptr + I), q1 = __ldg(agg_ptr + I + 1);
    T acc = T(0);
    int q = q0;
    for (; q + 4 <= q1; q += 4) {  // four independent loads in flight, added in member order
        const int m0 = __ldg(members + q), m1 = __ldg(members + q + 1);
        const int m2 = __ldg(members + q + 2), m3 = __ldg(members + q + 3);
        const T v0 = ld1<T, CG>(res + (size_t)m0 * b + d), v1 = ld1<T, CG>(res + (size_t)m1 * b + d);
        const T v2 = ld1<T, CG>(res + (size_t)m2 * b + d), v3 = ld1<T, CG>(res + (size_t)m3 * b + d);
        acc += v0;
        acc += v1;
        acc += v2;
        acc += v3;
    }
    for (; q < q1; ++q) acc += ld1<T, CG>(res + (size_t)__ldg(members + q) * b + d);
    rc[(size_t)I * b + d] = acc;
}

// ---------------------------------------------------------------------------
// one-step kernels
// ---------------------------------------------------------------------------
template <typename T, int B, int FB, bool FM>
__global__ void __launch_bounds__(256, 4) spmv_kernel(int n, const int* __restrict__ rp,
                                                   const int* __restrict__ ci,
                                                   const T* __restrict__ vals, const T* __restrict__ x,
                                                   const T* __restrict__ rhs, T* __restrict__ y) {
    const long i = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;  // uniform per warp
    spmv_row<T, B, FB, false, true, FM>(i, threadIdx.x & (kWarp - 1), rp, ci, vals, x, rhs, y);
}

template <typename T>
int launch_spmv(int b, int fb, int fm, int n, const int* rp, const int* ci, const T* vals, const T* x, const T* rhs,
                T* y, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    const int threads = 256;
    const int blocks = ceil_div((long)n * kWarp, threads);
    switch (b * 16 + fb) {
#define CASE(BB, FF) \
    case BB * 16 + FF:                                                                                      \
        if ((fm && HasFm<T, BB, FF>::value                                                                  \
                 ? launch_k(spmv_kernel<T, BB, FF, HasFm<T, BB, FF>::value>, blocks, threads, 0, s, n, rp, ci, vals, \
                            x, rhs, y)                                                                      \
                 : launch_k(spmv_kernel<T, BB, FF, false>, blocks, threads, 0, s, n, rp, ci, vals, x, rhs, y)) != \
            cudaSuccess)                                                                                    \
            return BAMG_ECUDA;                                                                              \
        break;
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_spmv<double>(int, int, int, int, const int*, const int*, const double*, const double*,
                                 const double*, double*, cudaStream_t);
template int launch_spmv<float>(int, int, int, int, const int*, const int*, const float*, const float*,
                                const float*, float*, cudaStream_t);

template <typename T>
__global__ void restrict_kernel(int b, int nc, const int* __restrict__ agg_ptr, const int* __restrict__ members,
                                const T* __restrict__ res, T* __restrict__ rc) {
    pdl_wait();
    pdl_trigger();
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (long)nc * b) restrict_dof<T, false>(t, b, agg_ptr, members, res, rc);
}

template <typename T>
int launch_restrict(int b, int nc, const int* agg_ptr, const int* members, const T* res, T* rc,
                    cudaStream_t s) {
    if (nc <= 0) return BAMG_OK;
    if (launch_k(restrict_kernel<T>, ceil_div((long)nc * b, 256), 256, 0, s, b, nc, agg_ptr, members, res, rc) !=
        cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}
template int launch_restrict<double>(int, int, const int*, const int*, const double*, double*, cudaStream_t);
template int launch_restrict<float>(int, int, const int*, const int*, const float*, float*, cudaStream_t);

// prolongation and correction u += P uc, P piecewise constant per dof
template <typename T>
__global__ void prolong_kernel(int b, int n, const int* __restrict__ agg, const T* __restrict__ uc,
                               T* __restrict__ u) {
    pdl_wait();
    pdl_trigger();
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(e / b);
    if (i >= n) return;
    const int d = (int)(e - (long)i * b);
    u[e] += uc[(size_t)agg[i] * b + d];
}

// the nodes of a range that a field step leaves alone: y = x (+ P uc), or
// zero without x (the zero initial guess)
template <typename T>
__global__ void copy_prolong_kernel(int b, int n, const int* __restrict__ agg, const T* __restrict__ x,
                                    const T* __restrict__ uc, T* __restrict__ y) {
    pdl_wait();
    pdl_trigger();
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(e / b);
    if (i >= n) return;
    const int d = (int)(e - (long)i * b);
    T v = x ? x[e] : T(0);
    if (x && uc) v += uc[(size_t)agg[i] * b + d];
    y[e] = v;
}

template <typename T>
int launch_copy_prolong(int b, int n, const int* agg, const T* x, const T* uc, T* y, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    if (launch_k(copy_prolong_kernel<T>, ceil_div((long)n * b, 256), 256, 0, s, b, n, agg, x, uc, y) != cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}
template int launch_copy_prolong<double>(int, int, const int*, const double*, const double*, double*, cudaStream_t);
template int launch_copy_prolong<float>(int, int, const int*, const float*, const float*, float*, cudaStream_t);

template <typename T>
int launch_prolong(int b, int n, const int* agg, const T* uc, T* u, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    if (launch_k(prolong_kernel<T>, ceil_div((long)n * b, 256), 256, 0, s, b, n, agg, uc, u) != cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}
template int launch_prolong<double>(int, int, const int*, const double*, double*, cudaStream_t);
template int launch_prolong<float>(int, int, const int*, const float*, float*, cudaStream_t);

template <typename T, int B, int FB, bool FM>
__global__ void __launch_bounds__(256, 4) bgs_colour_kernel(BgsArgs a) {
    const long q = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= a.n_in_colour) return;  // uniform per warp
    bgs_node<T, B, FB, false, true, FM>(a, q, threadIdx.x & (kWarp - 1));
}

template <typename T>
int launch_bgs_colour(int b, int fb, const BgsArgs& a, cudaStream_t s) {
    if (a.n_in_colour <= 0) return BAMG_OK;
    const int threads = 256;
    const int blocks = ceil_div((long)a.n_in_colour * kWarp, threads);
    switch (b * 16 + fb) {
#define CASE(BB, FF) \
    case BB * 16 + FF:                                                                          \
        if ((a.fm && HasFm<T, BB, FF>::value                                                    \
                 ? launch_k(bgs_colour_kernel<T, BB, FF, HasFm<T, BB, FF>::value>, blocks, threads, 0, s, a) \
                 : launch_k(bgs_colour_kernel<T, BB, FF, false>, blocks, threads, 0, s, a)) != cudaSuccess) \
            return BAMG_ECUDA;                                                                  \
        break;
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_bgs_colour<double>(int, int, const BgsArgs&, cudaStream_t);
template int launch_bgs_colour<float>(int, int, const BgsArgs&, cudaStream_t);

// One colour of one field step with W warps per node, one node per CTA (the
// same arithmetic as bgs_node; row sums in another order): warp w takes the
// row's blocks w G + kk, w G + kk + W G, ... (G blocks per warp pass), the W
// partial row sums meet in shared memory in warp order, and warp 0 finishes
// the node.  W times shorter chains of dependent loads per node than one warp
// per node: for levels whose rows are long and whose colours are small.
template <typename T, int B, int FB, int W, bool FM>
__global__ void __launch_bounds__(W * 32) bgs_wide_kernel(BgsArgs a) {
    __shared__ T part[W][FB];
    const long q = blockIdx.x;
    if (q >= a.n_in_colour) return;  // whole CTA
    constexpr int G = kWarp / FB;  // blocks of the row per warp pass
    const int lane = threadIdx.x & (kWarp - 1), w = threadIdx.x >> 5;
    const int kk = lane / FB;
    const int r = lane - kk * FB;
    const int f0 = a.field * FB;
    const T* __restrict__ vals = static_cast<const T*>(a.vals);
    const T* x_in = static_cast<const T*>(a.x_in);
    const T* uc = static_cast<const T*>(a.uc);
    const T* xt = static_cast<const T*>(a.xt);
    const int i = __ldg(a.nodes + q);
    const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1);
    T drow[FB];
    if (w == 0 && lane < FB) {
        const T* D = static_cast<const T*>(a.dinv) + ((size_t)i * a.F + a.field) * FB * FB + (size_t)lane * FB;
#pragma unroll
        for (int c = 0; c < FB; ++c) drow[c] = __ldg(D + c);
    }
    // the lane's first block before the wait (as in bgs_node)
    const int kf = k0 + w * G + kk;
    const bool have = kk < G && kf < k1;
    const int kq = min(kf, k1 - 1);
    const int jf = __ldg(a.ci + kq);
    const bool lowf = __ldg(a.lowk + kq) != 0;
    const T* vb = vrow<T, B, FB, FM>(vals, k0, k1, k0, f0 + r);
    constexpr int VS = vstride<T, B, FB, FM>();
    T arf[B];
    if (x_in || lowf) load_row<T, B>(vb + (size_t)(kq - k0) * VS, arf);
    const int agf = (x_in && uc) ? __ldg(a.agg + jf) : 0;
    pdl_wait();
    pdl_trigger();
    const T bi = (w == 0 && lane < FB) ? static_cast<const T*>(a.rhs)[(size_t)i * B + f0 + lane] : T(0);
    T acc = T(0);
    if (have) bgs_walk<T, B, FB, false, W * G>(a, xt, x_in, uc, vb, VS, k0, kf, k1, jf, lowf, agf, arf, acc);
    acc = reduce_rows<T, FB>(acc, lane);
    if (lane < FB) part[w][lane] = acc;
    __syncthreads();
    if (w != 0) return;
    acc = T(0);
    if (lane < FB)
#pragma unroll
        for (int ww = 0; ww < W; ++ww) acc += part[ww][lane];
    T t = T(0);
    if (lane < FB) t = bi - acc;
    T xn = T(0);
#pragma unroll
    for (int c = 0; c < FB; ++c) {
        const T tc = __shfl_sync(0xffffffffu, t, c);
        if (lane < FB) xn = fma(drow[c], tc, xn);
    }
    if (lane < FB) static_cast<T*>(a.xt)[(size_t)i * FB + lane] = xn;
    const T xf = __shfl_sync(0xffffffffu, xn, (lane - f0) & (kWarp - 1));
    if (lane < B) {
        const size_t e = (size_t)i * B + lane;
        T v = x_in ? x_in[e] : T(0);
        if (x_in && uc) v += uc[(size_t)__ldg(a.agg + i) * B + lane];
        if (lane >= f0 && lane < f0 + FB) {
            const T om = a.omega_node ? static_cast<const T*>(a.omega_node)[(size_t)i * a.F + a.field] : T(a.omega);
            v = fma(om, xf, v);
        }
        static_cast<T*>(a.x_out)[e] = v;
    }
}

constexpr int kWideWarps = 4;

template <typename T>
int launch_bgs_colour_wide(int b, int fb, const BgsArgs& a, cudaStream_t s) {
    if (a.n_in_colour <= 0) return BAMG_OK;
    const int blocks = a.n_in_colour;
    switch (b * 16 + fb) {
#define CASE(BB, FF) \
    case BB * 16 + FF:                                                                                          \
        if ((a.fm && HasFm<T, BB, FF>::value                                                                    \
                 ? launch_k(bgs_wide_kernel<T, BB, FF, kWideWarps, HasFm<T, BB, FF>::value>, blocks, kWideWarps * 32, \
                            0, s, a)                                                                            \
                 : launch_k(bgs_wide_kernel<T, BB, FF, kWideWarps, false>, blocks, kWideWarps * 32, 0, s, a)) !=   \
            cudaSuccess)                                                                                        \
            return BAMG_ECUDA;                                                                                  \
        break;
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_bgs_colour_wide<double>(int, int, const BgsArgs&, cudaStream_t);
template int launch_bgs_colour_wide<float>(int, int, const BgsArgs&, cudaStream_t);

// lowk[k] for every block of row i: its column j != i has a lower colour
__global__ void lower_flags_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                   const int* __restrict__ colour, unsigned char* __restrict__ lowk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ci_ = colour[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        lowk[k] = (j != i && colour[j] < ci_) ? 1 : 0;
    }
}
int launch_lower_flags(int n, const int* rp, const int* ci, const int* colour, unsigned char* lowk, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    lower_flags_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, ci, colour, lowk);
    return launched(1);
}

template <typename T, typename S>
__global__ void dense_gemv_kernel(int nd, const S* __restrict__ ainv, const T* __restrict__ x,
                                  T* __restrict__ y) {
    pdl_wait();
    pdl_trigger();
    const int row = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (row >= nd) return;
    gemv_row<T, S, false>(row, threadIdx.x & 31, nd, ainv, x, y);
}

template <typename T, typename S>
int launch_dense_gemv(int nd, const S* ainv, const T* x, T* y, cudaStream_t s) {
    if (nd <= 0) return BAMG_OK;
    if (launch_k(dense_gemv_kernel<T, S>, ceil_div((long)nd * kWarp, 256), 256, 0, s, nd, ainv, x, y) !=
        cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}
template int launch_dense_gemv<double, double>(int, const double*, const double*, double*, cudaStream_t);
template int launch_dense_gemv<float, double>(int, const double*, const float*, float*, cudaStream_t);
template int launch_dense_gemv<float, float>(int, const float*, const float*, float*, cudaStream_t);
template int launch_dense_gemv<double, float>(int, const float*, const double*, double*, cudaStream_t);

// ---------------------------------------------------------------------------
// Thread-per-row variants for large levels.  One thread owns one scalar row
// and walks the blocks of its block row with the loop unrolled, so every
// thread keeps several block-row loads in flight (the warp-per-row mapping
// above keeps one short row per warp in flight, which leaves HBM idle on
// levels far larger than L2).  The setup autotuner picks the mapping per
// level and kernel by timing both.
// ---------------------------------------------------------------------------
// G lanes per scalar row, lane s taking blocks k0 + s, k0 + s + G, ... (G = 1:
// the whole row); the lanes' partial sums meet by shuffles (consecutive lanes
// of one warp).  G > 1 gives each warp fewer, longer contiguous runs of a
// row's blocks and each lane a shorter chain of dependent loads.
template <typename T, int B, int FB, bool FM, int G>
__global__ void __launch_bounds__(256) spmv_tpr_kernel(int n, const int* __restrict__ rp,
                                                       const int* __restrict__ ci, const T* __restrict__ vals,
                                                       const T* __restrict__ x, const T* __restrict__ rhs,
                                                       T* __restrict__ y) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long row = t / G;  // scalar row i * B + r
    const int sl = (int)(t - row * G);
    const int i = (int)(row / B);
    const bool act = i < n;
    if (G == 1 && !act) return;
    const int r = (int)(row - (long)i * B);
    T acc = T(0);
    if (act) {
        const int k0 = __ldg(rp + i), k1 = __ldg(rp + i + 1);
        const int kf = k0 + sl;
        // the first block before the wait (fixed for the cycle)
        int jf = 0;
        T af[B];
        if (kf < k1) {
            jf = __ldg(ci + kf);
            load_row<T, B>(vrow<T, B, FB, FM>(vals, k0, k1, kf, r), af);
        }
        pdl_wait();
        pdl_trigger();
        if (kf < k1) {
            T xv[B];
            load_row<T, B>(x + (size_t)jf * B, xv);
#pragma unroll
            for (int c = 0; c < B; ++c) acc = fma(af[c], xv[c], acc);
        }
#pragma unroll 4
        for (int k = kf + G; k < k1; k += G) {
            const int j = __ldg(ci + k);
            T a[B], xv[B];
            load_row<T, B>(vrow<T, B, FB, FM>(vals, k0, k1, k, r), a);
            load_row<T, B>(x + (size_t)j * B, xv);
#pragma unroll
            for (int c = 0; c < B; ++c) acc = fma(a[c], xv[c], acc);
        }
    }
    if constexpr (G > 1) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (!act || sl != 0) return;
    }
    y[(size_t)i * B + r] = rhs ? rhs[(size_t)i * B + r] - acc : acc;
}

template <typename T>
int launch_spmv_tpr(int b, int fb, int fm, int n, const int* rp, const int* ci, const T* vals, const T* x,
                    const T* rhs, T* y, cudaStream_t s, int variant) {
    if (n <= 0) return BAMG_OK;
    const int G = variant == 1 ? 4 : 1;
    const int blocks = ceil_div((long)n * b * G, 256);
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                         \
    case BB * 16 + FF: {                                                                                     \
        constexpr bool kFm = HasFm<T, BB, FF>::value;                                                       \
        cudaError_t e;                                                                                       \
        if (G == 4)                                                                                          \
            e = (fm && kFm) ? launch_k(spmv_tpr_kernel<T, BB, FF, kFm, 4>, blocks, 256, 0, s, n, rp, ci, vals, \
                                       x, rhs, y)                                                            \
                            : launch_k(spmv_tpr_kernel<T, BB, FF, false, 4>, blocks, 256, 0, s, n, rp, ci,   \
                                       vals, x, rhs, y);                                                     \
        else                                                                                                 \
            e = (fm && kFm) ? launch_k(spmv_tpr_kernel<T, BB, FF, kFm, 1>, blocks, 256, 0, s, n, rp, ci, vals, \
                                       x, rhs, y)                                                            \
                            : launch_k(spmv_tpr_kernel<T, BB, FF, false, 1>, blocks, 256, 0, s, n, rp, ci,   \
                                       vals, x, rhs, y);                                                     \
        if (e != cudaSuccess) return BAMG_ECUDA;                                                             \
        break;                                                                                               \
    }
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_spmv_tpr<double>(int, int, int, int, const int*, const int*, const double*, const double*,
                                     const double*, double*, cudaStream_t, int);
template int launch_spmv_tpr<float>(int, int, int, int, const int*, const int*, const float*, const float*,
                                    const float*, float*, cudaStream_t, int);

// Residual after one pre-smoothing sweep from a zero iterate with one field
// (F = 1) and one damping value: the sweep left x = omega x~ and, for every
// node i, A_ii x~_i = b_i - sum over lower-colour j of A_ij x~_j (the
// multicolour Gauss-Seidel step of Algorithm 1), so
//   (b - A x)_i = (1 - omega) b_i - omega sum over higher-colour j of A_ij x~_j
// (nodes of one colour do not couple): only the blocks of higher colour are
// read, about half of the row.  Thread per scalar row.
template <typename T, int B, bool FM>
__global__ void __launch_bounds__(256) residual_upper_kernel(int n, const int* __restrict__ rp,
                                                             const int* __restrict__ ci,
                                                             const unsigned char* __restrict__ lowk,
                                                             const T* __restrict__ vals, const T* __restrict__ xt,
                                                             const T* __restrict__ rhs, T omega, T* __restrict__ y) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / B);
    if (i >= n) return;
    const int r = (int)(t - (long)i * B);
    const int k0 = __ldg(rp + i), k1 = __ldg(rp + i + 1);
    pdl_wait();
    pdl_trigger();
    T acc = T(0);
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
        const int j = __ldg(ci + k);
        if (j == i || __ldg(lowk + k)) continue;
        T a[B], xv[B];
        load_row<T, B>(vrow<T, B, B, FM>(vals, k0, k1, k, r), a);
        load_row<T, B>(xt + (size_t)j * B, xv);
#pragma unroll
        for (int c = 0; c < B; ++c) acc = fma(a[c], xv[c], acc);
    }
    const size_t e = (size_t)i * B + r;
    y[e] = (T(1) - omega) * rhs[e] - omega * acc;
}

// (one field: the values are block-major, fm is unused)
template <typename T>
int launch_residual_upper(int b, int fm, int n, const int* rp, const int* ci, const unsigned char* lowk,
                          const T* vals, const T* xt, const T* rhs, double omega, T* y, cudaStream_t s) {
    (void)fm;
    if (n <= 0) return BAMG_OK;
    const int blocks = ceil_div((long)n * b, 256);
    cudaError_t e = cudaErrorInvalidValue;
    switch (b) {
#define CASE(BB)                                                                                          \
    case BB:                                                                                              \
        e = launch_k(residual_upper_kernel<T, BB, false>, blocks, 256, 0, s, n, rp, ci, lowk, vals, xt, rhs, \
                     (T)omega, y);                                                                        \
        break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    if (e != cudaSuccess) return BAMG_ECUDA;
    return launched(1);
}
template int launch_residual_upper<double>(int, int, int, const int*, const int*, const unsigned char*,
                                           const double*, const double*, const double*, double, double*,
                                           cudaStream_t);
template int launch_residual_upper<float>(int, int, int, const int*, const int*, const unsigned char*, const float*,
                                          const float*, const float*, double, float*, cudaStream_t);

// threads per CTA: a multiple of both FB and the warp size (the launch may use
// half of it: smaller CTAs spread a small colour over more SMs)
template <int FB>
struct TprBlock {
    static constexpr int kThreads = RowThreads<FB>::kThreads;
};

// One colour of one field step (same arithmetic as bgs_node up to the order
// of the row sum), G * FB threads per node: the G consecutive lanes of scalar
// row r take every G-th block of the row (G = 1: the whole row), their
// partial sums meet by a shuffle, and the FB row sums in shared memory for
// the inverse.  G > 1 shortens each thread's chain of index-then-gather loads
// (one block row after another), the latency that bounds large colours.
template <typename T, int B, int FB, int G, bool FM>
__global__ void __launch_bounds__(TprBlock<FB>::kThreads) bgs_tpr_kernel(BgsArgs a) {
    __shared__ T sh_t[TprBlock<FB>::kThreads];
    const int tloc = threadIdx.x;
    const int nloc = tloc / (FB * G);
    const int w = tloc - nloc * (FB * G);
    const int r = w / G, sl = w - r * G;  // scalar row, slice of the row's blocks
    const long q = (long)blockIdx.x * (blockDim.x / (FB * G)) + nloc;
    const bool act = q < a.n_in_colour;
    const int f0 = a.field * FB;
    const T* __restrict__ vals = static_cast<const T*>(a.vals);
    const T* __restrict__ x_in = static_cast<const T*>(a.x_in);
    const T* __restrict__ uc = static_cast<const T*>(a.uc);
    const T* __restrict__ xt = static_cast<const T*>(a.xt);
    int i = 0;
    T t = T(0);
    T acc = T(0);
    if (act) {
        i = __ldg(a.nodes + q);
        const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1);
        // the first block's static loads before the wait (as in bgs_node)
        const int kf = k0 + sl;
        const bool have = kf < k1;
        const int kq = min(kf, k1 - 1);  // rows hold their diagonal block
        const int jf = __ldg(a.ci + kq);
        const bool lowf = __ldg(a.lowk + kq) != 0;
        const T* vb = vrow<T, B, FB, FM>(vals, k0, k1, k0, f0 + r);
        constexpr int VS = vstride<T, B, FB, FM>();
        T arf[B];
        if (x_in || lowf) load_row<T, B>(vb + (size_t)(kq - k0) * VS, arf);
        const int agf = (x_in && uc) ? __ldg(a.agg + jf) : 0;
        pdl_wait();
        pdl_trigger();
        if (have) {
            // (a plain loop: the software-pipelined walk of bgs_node needs
            // more registers, and at this mapping's occupancy that measured
            // slower on levels far larger than L2)
            bgs_block<T, B, FB, false>(a, xt, x_in, uc, jf, arf, lowf, agf, acc);
#pragma unroll(G > 1 ? 8 : 4)
            for (int k = kf + G; k < k1; k += G) {
                const bool lower = __ldg(a.lowk + k) != 0;
                if (!x_in && !lower) continue;
                const int j = __ldg(a.ci + k);
                T arow[B];
                load_row<T, B>(vb + (size_t)(k - k0) * VS, arow);
                bgs_block<T, B, FB, false>(a, xt, x_in, uc, j, arow, lower, (x_in && uc) ? __ldg(a.agg + j) : 0,
                                           acc);
            }
        }
    }
    if constexpr (G > 1) {  // the G slices of a row are consecutive lanes of one warp
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    }
    if (act && sl == 0) t = static_cast<const T*>(a.rhs)[(size_t)i * B + f0 + r] - acc;
    if (sl == 0) sh_t[nloc * FB + r] = t;
    __syncthreads();
    if (!act || sl != 0) return;
    const T* D = static_cast<const T*>(a.dinv) + ((size_t)i * a.F + a.field) * FB * FB + (size_t)r * FB;
    T xn = T(0);
#pragma unroll
    for (int c = 0; c < FB; ++c) xn = fma(__ldg(D + c), sh_t[nloc * FB + c], xn);
    static_cast<T*>(a.xt)[(size_t)i * FB + r] = xn;
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
int launch_bgs_colour_tpr(int b, int fb, const BgsArgs& a, cudaStream_t s, int variant) {
    if (a.n_in_colour <= 0) return BAMG_OK;
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                          \
    case BB * 16 + FF: {                                                                                      \
        const int threads = TprBlock<FF>::kThreads >> (variant == 1 ? 1 : 0);                                 \
        constexpr bool kFm = HasFm<T, BB, FF>::value;                                                        \
        const int g4 = ceil_div(a.n_in_colour, threads / (FF * 4)), g1 = ceil_div(a.n_in_colour, threads / FF); \
        cudaError_t e;                                                                                        \
        if (variant == 2)                                                                                     \
            e = (a.fm && kFm) ? launch_k(bgs_tpr_kernel<T, BB, FF, 4, kFm>, g4, threads, 0, s, a)              \
                              : launch_k(bgs_tpr_kernel<T, BB, FF, 4, false>, g4, threads, 0, s, a);           \
        else                                                                                                  \
            e = (a.fm && kFm) ? launch_k(bgs_tpr_kernel<T, BB, FF, 1, kFm>, g1, threads, 0, s, a)              \
                              : launch_k(bgs_tpr_kernel<T, BB, FF, 1, false>, g1, threads, 0, s, a);           \
        if (e != cudaSuccess) return BAMG_ECUDA;                                                              \
        break;                                                                                                \
    }
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_bgs_colour_tpr<double>(int, int, const BgsArgs&, cudaStream_t, int);
template int launch_bgs_colour_tpr<float>(int, int, const BgsArgs&, cudaStream_t, int);

// One colour of one field step (same arithmetic as bgs_node up to the order of
// the row sums) with G lanes per node, each lane taking whole blocks: lane s
// takes blocks k0 + s, k0 + s + G, ... and loads the block's FB field rows as
// independent vector loads, so each lane has several loads in flight (the
// four-lanes-per-row mapping has one row load per lane at a time, which
// bounds large colours by latency).  The FB row sums of the G lanes meet by
// shuffles within the lane group; lane r < FB finishes row r.  Blocks of
// higher colour contribute x_in only; x~ is loaded for every block when x_in
// is set (no branch on the colour flag before the gathers) and used where the
// flag is set.  XIN: x_in is set.  FB x B <= 16 (the block in registers).
template <typename T, int B, int FB, int G, bool FM, bool XIN>
__device__ __forceinline__ void bsp_body(const BgsArgs& a, bool act, long q, int s) {
    static_assert(32 % G == 0, "lane groups inside a warp");
    const int f0 = a.field * FB;
    const T* __restrict__ vals = static_cast<const T*>(a.vals);
    const T* __restrict__ x_in = static_cast<const T*>(a.x_in);
    const T* __restrict__ uc = static_cast<const T*>(a.uc);
    const T* xt = static_cast<const T*>(a.xt);
    T acc[FB];
#pragma unroll
    for (int r = 0; r < FB; ++r) acc[r] = T(0);
    int i = 0;
    if (act) {
        i = __ldg(a.nodes + q);
        const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1);
        // the FB field rows of block k: FB * B contiguous values at vb + (k - k0) VS
        const T* vb = vrow<T, B, FB, FM>(vals, k0, k1, k0, f0);
        constexpr int VS = vstride<T, B, FB, FM>();
        pdl_wait();
        pdl_trigger();
#pragma unroll 2
        for (int k = k0 + s; k < k1; k += G) {
            const int j = __ldg(a.ci + k);
            const bool low = __ldg(a.lowk + k) != 0;  // j precedes i in the colour order
            if (!XIN && !low) continue;
            T ar[FB][B];
#pragma unroll
            for (int r = 0; r < FB; ++r) load_row<T, B>(vb + (size_t)(k - k0) * VS + r * B, ar[r]);
            T tv[FB];
            load_row<T, FB>(xt + (size_t)j * FB, tv);
            if constexpr (XIN) {
                T xv[B];
                load_row<T, B>(x_in + (size_t)j * B, xv);
                if (uc) {
                    T pv[B];
                    load_row<T, B>(uc + (size_t)__ldg(a.agg + j) * B, pv);
#pragma unroll
                    for (int c = 0; c < B; ++c) xv[c] += pv[c];
                }
#pragma unroll
                for (int r = 0; r < FB; ++r)
#pragma unroll
                    for (int c = 0; c < B; ++c) acc[r] = fma(ar[r][c], xv[c], acc[r]);
            }
#pragma unroll
            for (int r = 0; r < FB; ++r)
#pragma unroll
                for (int c = 0; c < FB; ++c) {
                    // column f0 + c of the row, by selects over register indices
                    T av = ar[r][c];
#pragma unroll
                    for (int ff = 1; ff < B / FB; ++ff) av = (ff == a.field) ? ar[r][ff * FB + c] : av;
                    const T nv = fma(av, tv[c], acc[r]);
                    acc[r] = low ? nv : acc[r];
                }
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < FB; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (!act || s >= FB) return;
    const T* rhs = static_cast<const T*>(a.rhs) + (size_t)i * B + f0;
    const T* D = static_cast<const T*>(a.dinv) + ((size_t)i * a.F + a.field) * FB * FB + (size_t)s * FB;
    T xn = T(0);
#pragma unroll
    for (int c = 0; c < FB; ++c) xn = fma(__ldg(D + c), rhs[c] - acc[c], xn);
    static_cast<T*>(a.xt)[(size_t)i * FB + s] = xn;
    T* __restrict__ x_out = static_cast<T*>(a.x_out);
    const T om = a.omega_node ? static_cast<const T*>(a.omega_node)[(size_t)i * a.F + a.field] : T(a.omega);
    const int ag = (XIN && uc) ? __ldg(a.agg + i) : 0;
    for (int m = 0; m < a.F; ++m) {
        const size_t e = (size_t)i * B + m * FB + s;
        T v = XIN ? x_in[e] : T(0);
        if (XIN && uc) v += uc[(size_t)ag * B + m * FB + s];
        if (m == a.field) v = fma(om, xn, v);
        x_out[e] = v;
    }
}

template <typename T, int B, int FB, int G, bool FM>
__global__ void __launch_bounds__(256) bgs_bsp_kernel(BgsArgs a) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long q = t / G;
    const int s = (int)(t - q * G);
    const bool act = q < a.n_in_colour;
    if (a.x_in) bsp_body<T, B, FB, G, FM, true>(a, act, q, s);
    else bsp_body<T, B, FB, G, FM, false>(a, act, q, s);
}

bool bsp_supported(int b, int fb) { return fb * b <= 16; }

template <typename T>
int launch_bgs_colour_bsp(int b, int fb, const BgsArgs& a, int G, cudaStream_t s) {
    if (!bsp_supported(b, fb) || (G != 8 && G != 16)) return BAMG_EUNSUPPORTED;
    if (a.n_in_colour <= 0) return BAMG_OK;
    const int grid = ceil_div((long)a.n_in_colour * G, 256);
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                        \
    case BB * 16 + FF: {                                                                                    \
        if constexpr (FF * BB <= 16) {                                                                      \
            constexpr bool kFm = HasFm<T, BB, FF>::value;                                                  \
            cudaError_t e;                                                                                  \
            if (G == 16)                                                                                    \
                e = (a.fm && kFm) ? launch_k(bgs_bsp_kernel<T, BB, FF, 16, kFm>, grid, 256, 0, s, a)        \
                                  : launch_k(bgs_bsp_kernel<T, BB, FF, 16, false>, grid, 256, 0, s, a);     \
            else                                                                                            \
                e = (a.fm && kFm) ? launch_k(bgs_bsp_kernel<T, BB, FF, 8, kFm>, grid, 256, 0, s, a)         \
                                  : launch_k(bgs_bsp_kernel<T, BB, FF, 8, false>, grid, 256, 0, s, a);      \
            if (e != cudaSuccess) return BAMG_ECUDA;                                                        \
            break;                                                                                          \
        } else {                                                                                            \
            return BAMG_EUNSUPPORTED;                                                                       \
        }                                                                                                   \
    }
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_bgs_colour_bsp<double>(int, int, const BgsArgs&, int, cudaStream_t);
template int launch_bgs_colour_bsp<float>(int, int, const BgsArgs&, int, cudaStream_t);

// One colour of one of several sweeps of the multicolour Gauss-Seidel
// sub-solve A_ff x~ = r_f of a field step (Algorithm 1 with the sub-solve
// iterated), one thread per scalar row of field f:
//   x~_i = D_i^{-1} (r_f,i - sum_{j != i} A_ff(i,j) x~_j)
// where, in the first sweep, a neighbour of higher colour contributes nothing
// (x~ starts from zero; its entry in xt is stale) and, in the later sweeps,
// its value from the previous sweep.  The nodes of one colour do not couple,
// so xt is read at other colours' nodes only and written at this colour's.
// rf (n x FB) holds r_f = b_f - A_f* x_in for every node, formed before the
// first sweep.  The last sweep also writes node i of x_out: x_in (+ P uc)
// with field f increased by omega x~_i.
template <typename T, int B, int FB, bool FM>
__global__ void __launch_bounds__(TprBlock<FB>::kThreads)
    gs_inner_kernel(BgsArgs a, const T* __restrict__ rf, int first, int last) {
    __shared__ T sh_t[TprBlock<FB>::kThreads];
    const int tloc = threadIdx.x;
    const int nloc = tloc / FB, r = tloc - nloc * FB;
    const long q = (long)blockIdx.x * (blockDim.x / FB) + nloc;
    const bool act = q < a.n_in_colour;
    const int f0 = a.field * FB;
    const T* __restrict__ vals = static_cast<const T*>(a.vals);
    T* xt = static_cast<T*>(a.xt);
    int i = 0;
    T t = T(0);
    if (act) {
        i = __ldg(a.nodes + q);
        const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1);
        // columns f0.. of scalar row f0 + r in each block of the row
        const T* vb = vrow<T, B, FB, FM>(vals, k0, k1, k0, f0 + r) + f0;
        constexpr int VS = vstride<T, B, FB, FM>();
        pdl_wait();
        pdl_trigger();
        T acc = T(0);
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            if (first && __ldg(a.lowk + k) == 0) continue;  // also skips the diagonal block
            const int j = __ldg(a.ci + k);
            if (j == i) continue;
            const T* ap = vb + (size_t)(k - k0) * VS;
            const T* xp = xt + (size_t)j * FB;
#pragma unroll
            for (int c = 0; c < FB; ++c) acc = fma(__ldg(ap + c), xp[c], acc);
        }
        t = rf[(size_t)i * FB + r] - acc;
    }
    sh_t[tloc] = t;
    __syncthreads();
    if (!act) return;
    const T* D = static_cast<const T*>(a.dinv) + ((size_t)i * a.F + a.field) * FB * FB + (size_t)r * FB;
    T xn = T(0);
#pragma unroll
    for (int c = 0; c < FB; ++c) xn = fma(__ldg(D + c), sh_t[nloc * FB + c], xn);
    xt[(size_t)i * FB + r] = xn;
    if (!last) return;
    const T* __restrict__ x_in = static_cast<const T*>(a.x_in);
    const T* __restrict__ uc = static_cast<const T*>(a.uc);
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
int launch_gs_inner(int b, int fb, const BgsArgs& a, const T* rf, bool first, bool last, cudaStream_t s) {
    if (a.n_in_colour <= 0) return BAMG_OK;
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                          \
    case BB * 16 + FF: {                                                                                      \
        const int threads = TprBlock<FF>::kThreads;                                                           \
        constexpr bool kFm = HasFm<T, BB, FF>::value;                                                        \
        const int grid = ceil_div(a.n_in_colour, threads / FF);                                               \
        const cudaError_t e =                                                                                 \
            (a.fm && kFm) ? launch_k(gs_inner_kernel<T, BB, FF, kFm>, grid, threads, 0, s, a, rf, (int)first, \
                                     (int)last)                                                               \
                          : launch_k(gs_inner_kernel<T, BB, FF, false>, grid, threads, 0, s, a, rf,          \
                                     (int)first, (int)last);                                                  \
        if (e != cudaSuccess) return BAMG_ECUDA;                                                              \
        break;                                                                                                \
    }
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_gs_inner<double>(int, int, const BgsArgs&, const double*, bool, bool, cudaStream_t);
template int launch_gs_inner<float>(int, int, const BgsArgs&, const float*, bool, bool, cudaStream_t);

// ---------------------------------------------------------------------------
// Tail kernel: one thread-block cluster executes a recorded list of V-cycle
// phases (every colour of every field step, residuals, restrictions, the
// coarsest solve and the post-smoothing with the fused prolongation) for the
// levels below a given one.  Inside a phase the work items are spread over
// all warps (or threads) of the cluster; between phases the cluster barrier
// (barrier.cluster arrive.release / wait.acquire) orders the global-memory
// writes of one phase before the reads of the next, and the reads of data
// written inside the launch bypass L1 (ld.global.cg).  Every thread executes
// every phase and every barrier (no early exit), so the hardware barrier
// never waits for a thread that has left.
// ---------------------------------------------------------------------------
// one recorded phase over the work items of the calling thread: warp w of W
// warps (gw), thread t of NT threads (gt)
template <typename T, int B, int FB>
__device__ __forceinline__ void run_phase(const TailPhase& ph, int lane, long gw, long W, long gt, long NT) {
    switch (ph.type) {
        case kPhaseBgs:
            if (HasFm<T, B, FB>::value && ph.bgs.fm)
                for (long q = gw; q < ph.n; q += W)
                    bgs_node<T, B, FB, true, false, HasFm<T, B, FB>::value>(ph.bgs, q, lane);
            else
                for (long q = gw; q < ph.n; q += W) bgs_node<T, B, FB, true>(ph.bgs, q, lane);
            break;
        case kPhaseResidual:
            if (HasFm<T, B, FB>::value && ph.fm)
                for (long i = gw; i < ph.n; i += W)
                    spmv_row<T, B, FB, true, false, HasFm<T, B, FB>::value>(
                        i, lane, ph.rp, ph.ci, static_cast<const T*>(ph.vals), static_cast<const T*>(ph.x),
                        static_cast<const T*>(ph.rhs), static_cast<T*>(ph.y));
            else
                for (long i = gw; i < ph.n; i += W)
                    spmv_row<T, B, FB, true>(i, lane, ph.rp, ph.ci, static_cast<const T*>(ph.vals),
                                             static_cast<const T*>(ph.x), static_cast<const T*>(ph.rhs),
                                             static_cast<T*>(ph.y));
            break;
        case kPhaseRestrict:
            for (long t = gt; t < (long)ph.n * B; t += NT)
                restrict_dof<T, true>(t, B, ph.rp, ph.ci, static_cast<const T*>(ph.x), static_cast<T*>(ph.y));
            break;
        case kPhaseGemv:
            for (long row = gw; row < ph.n; row += W)
                gemv_row<T, double, true>((int)row, lane, ph.n, static_cast<const double*>(ph.vals),
                                          static_cast<const T*>(ph.x), static_cast<T*>(ph.y));
            break;
        case kPhaseGemv32:
            for (long row = gw; row < ph.n; row += W)
                gemv_row<T, float, true>((int)row, lane, ph.n, static_cast<const float*>(ph.vals),
                                         static_cast<const T*>(ph.x), static_cast<T*>(ph.y));
            break;
        case kPhaseProlongCopy:  // y = x + P uc over n fine nodes (x may equal y); uc in rhs, agg in ci
            for (long e = gt; e < (long)ph.n * B; e += NT) {
                const int i = (int)(e / B), d = (int)(e - (long)i * B);
                static_cast<T*>(ph.y)[e] =
                    ld1<T, true>(static_cast<const T*>(ph.x) + e) +
                    ld1<T, true>(static_cast<const T*>(ph.rhs) + (size_t)__ldg(ph.ci + i) * B + d);
            }
            break;
        case kPhaseZero:
            for (long e = gt; e < (long)ph.n * B; e += NT) static_cast<T*>(ph.y)[e] = T(0);
            break;
        default:
            break;
    }
}

template <typename T, int B, int FB>
__global__ void __launch_bounds__(kTailThreads, 1) tail_kernel(const TailPhase* __restrict__ phases, int nphase) {
    cg::cluster_group cl = cg::this_cluster();
    const int lane = threadIdx.x & (kWarp - 1);
    const int warps_per_cta = blockDim.x >> 5;
    const long gw = (long)cl.block_rank() * warps_per_cta + (threadIdx.x >> 5);
    const long W = (long)cl.num_blocks() * warps_per_cta;
    const long gt = (long)cl.block_rank() * blockDim.x + threadIdx.x;
    const long NT = (long)cl.num_blocks() * blockDim.x;
    for (int p = 0; p < nphase; ++p) {
        run_phase<T, B, FB>(phases[p], lane, gw, W, gt, NT);
        cl.sync();
    }
}

// ---------------------------------------------------------------------------
// Grid tail: the same recorded phases executed by every CTA of a cooperative
// launch (all SMs), with the bounded grid barrier between phases.  Writes of
// one phase reach L2 before the barrier (the barrier fences) and the next
// phase reads data written inside the launch through L2 (ld.global.cg).  A
// CTA whose barrier wait ran out leaves; every other CTA then runs out at its
// own next barrier, so the launch ends with kDevTimeout set.
// ---------------------------------------------------------------------------
template <typename T, int B, int FB>
__global__ void __launch_bounds__(kTailThreads, 1) grid_tail_kernel(const TailPhase* __restrict__ phases, int nphase,
                                                                    unsigned* bar, int* err) {
    const int lane = threadIdx.x & (kWarp - 1);
    const int warps_per_cta = blockDim.x >> 5;
    const long gw = (long)blockIdx.x * warps_per_cta + (threadIdx.x >> 5);
    const long W = (long)gridDim.x * warps_per_cta;
    const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long NT = (long)gridDim.x * blockDim.x;
    for (int p = 0; p < nphase; ++p) {
        run_phase<T, B, FB>(phases[p], lane, gw, W, gt, NT);
        if (!grid_barrier(bar, err)) return;
    }
}

template <typename T, int B, int FB>
static int launch_grid_tail_t(const TailPhase* phases, int nphase, int grid, unsigned* bar, int* err,
                              cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(kTailThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BAMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, grid_tail_kernel<T, B, FB>, phases, nphase, bar, err));
    return launched(1);
}

template <typename T, int B, int FB>
static int grid_tail_size_t() {
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grid_tail_kernel<T, B, FB>, kTailThreads, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms * per_sm;
}

template <typename T>
int launch_grid_tail(int b, int fb, const TailPhase* phases, int nphase, int grid, unsigned* bar, int* err,
                     cudaStream_t s) {
    switch (b * 16 + fb) {
#define CASE(BB, FF) \
    case BB * 16 + FF: return launch_grid_tail_t<T, BB, FF>(phases, nphase, grid, bar, err, s);
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
}
template int launch_grid_tail<double>(int, int, const TailPhase*, int, int, unsigned*, int*, cudaStream_t);
template int launch_grid_tail<float>(int, int, const TailPhase*, int, int, unsigned*, int*, cudaStream_t);

template <typename T>
int grid_tail_size(int b, int fb) {
    switch (b * 16 + fb) {
#define CASE(BB, FF) \
    case BB * 16 + FF: return grid_tail_size_t<T, BB, FF>();
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return 0;
    }
}
template int grid_tail_size<double>(int, int);
template int grid_tail_size<float>(int, int);

static void fill_cluster_config(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr, int cluster, cudaStream_t s) {
    *cfg = cudaLaunchConfig_t{};
    cfg->gridDim = dim3((unsigned)cluster, 1, 1);
    cfg->blockDim = dim3(kTailThreads, 1, 1);
    cfg->dynamicSmemBytes = 0;
    cfg->stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg->attrs = attr;
    cfg->numAttrs = 1;
}

template <typename T, int B, int FB>
static int launch_tail_t(const TailPhase* phases, int nphase, int cluster, cudaStream_t s) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    fill_cluster_config(&cfg, attr, cluster, s);
    BAMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, tail_kernel<T, B, FB>, phases, nphase));
    return launched(1);
}

// largest cluster size <= want (a power of two) that can be resident
template <typename T, int B, int FB>
static int tail_cluster_size_t(int want) {
    if (cudaFuncSetAttribute(tail_kernel<T, B, FB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess) {
        cudaGetLastError();
        if (want > 8) want = 8;
    }
    for (int c = want; c >= 1; c >>= 1) {
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute attr[1];
        fill_cluster_config(&cfg, attr, c, nullptr);
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, tail_kernel<T, B, FB>, &cfg) == cudaSuccess && clusters >= 1)
            return c;
        cudaGetLastError();
    }
    return 0;
}

template <typename T>
int launch_tail(int b, int fb, const TailPhase* phases, int nphase, int cluster, cudaStream_t s) {
    switch (b * 16 + fb) {
#define CASE(BB, FF) \
    case BB * 16 + FF: return launch_tail_t<T, BB, FF>(phases, nphase, cluster, s);
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
}
template int launch_tail<double>(int, int, const TailPhase*, int, int, cudaStream_t);
template int launch_tail<float>(int, int, const TailPhase*, int, int, cudaStream_t);

template <typename T>
int tail_cluster_size(int b, int fb, int want) {
    switch (b * 16 + fb) {
#define CASE(BB, FF) \
    case BB * 16 + FF: return tail_cluster_size_t<T, BB, FF>(want);
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return 0;
    }
}
template int tail_cluster_size<double>(int, int, int);
template int tail_cluster_size<float>(int, int, int);

// ---------------------------------------------------------------------------
// precision casts at the cycle boundary (FP64 Krylov vectors <-> FP32 cycle)
// ---------------------------------------------------------------------------
__global__ void cast_d2f_kernel(long m, const double* __restrict__ x, float* __restrict__ y) {
    pdl_wait();
    pdl_trigger();
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (long)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
}
__global__ void cast_f2d_kernel(long m, const float* __restrict__ x, double* __restrict__ y) {
    pdl_wait();
    pdl_trigger();
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (long)gridDim.x * blockDim.x)
        y[e] = (double)x[e];
}
static int grid_for(long m) {
    long g = (m + 255) / 256;
    return (int)(g < 152L * 16 ? (g > 0 ? g : 1) : 152L * 16);
}
int launch_cast_d2f(long m, const double* x, float* y, cudaStream_t s) {
    if (m <= 0) return BAMG_OK;
    if (launch_k(cast_d2f_kernel, grid_for(m), 256, 0, s, m, x, y) != cudaSuccess) return BAMG_ECUDA;
    return launched(1);
}
int launch_cast_f2d(long m, const float* x, double* y, cudaStream_t s) {
    if (m <= 0) return BAMG_OK;
    if (launch_k(cast_f2d_kernel, grid_for(m), 256, 0, s, m, x, y) != cudaSuccess) return BAMG_ECUDA;
    return launched(1);
}

}  // namespace bamg
