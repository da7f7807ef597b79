// FP64 kernels of the outer flexible GMRES: Arnoldi orthogonalisation by
// classical Gram-Schmidt applied twice (CGS2), Givens rotations of the
// Hessenberg column, the triangular solve for y and the update x += Z y.
// (The paper applies its V-cycle inside GMRES: Sec. 3 and Sec. 5.1.)
//
// Reductions are deterministic: every vector is cut into the same fixed
// chunks (one CTA each), every chunk reduces in a fixed tree, and the sums
// of the chunk partials are formed in chunk order by the last CTA to finish
// (it takes a ticket with an atomic after a memory fence; no CTA waits for
// another).  The Givens update of the Hessenberg column runs in that same
// last CTA of the final reduction of an Arnoldi step.
#include <math.h>

#include "common.cuh"

namespace bamg {

constexpr int kKThreads = 256;
constexpr int kDotGroup = 16;  // dot products accumulated together per pass
// ||w1||^2 / ||w||^2 below which an Arnoldi step projects a second time
// (eta = 0.01: the first projection removed more than 99.99% of ||w||^2)
constexpr double kReorthRatio = 1e-4;

// fixed chunking of a vector of length N: at least 256 elements per chunk, at
// most two CTAs per SM of the GB300 (152 SMs).  The basis vectors are mostly
// L2-resident and the rate is set by the loads in flight across the GPU:
// measured on the solves here, 2048-element chunks (fewer CTAs) and four CTAs
// per SM (more block sums and partials) were both slower.
int krylov_chunks(long N) {
    long c = (N + 255) / 256;
    if (c > 2 * 152) c = 2 * 152;
    return (int)(c < 1 ? 1 : c);
}

__device__ __forceinline__ void chunk_range(long N, long* e0, long* e1) {
    const long per = (N + gridDim.x - 1) / gridDim.x;
    *e0 = (long)blockIdx.x * per;
    *e1 = min(N, *e0 + per);
}

// Dots of x with G vectors over the chunk (G fixed at compile time, so every
// issued FMA is a useful one: the FP64 pipe, 2 FMA per clock per SM on
// GB300, bounds these passes): vector g is Y_{v0+g}, or x itself for the last
// one when xx is set.  The block sums go to partial[(v0 + g) * nchunk + chunk].
template <int G>
__device__ __forceinline__ void chunk_dots_fixed(long e0, long e1, const double* __restrict__ x,
                                                 const double* __restrict__ Y, long ld, int v0, bool xx,
                                                 double* __restrict__ partial, double* sh) {
    const double* yp[G];
#pragma unroll
    for (int g = 0; g < G; ++g) yp[g] = (xx && g == G - 1) ? x : Y + (size_t)(v0 + g) * ld;
    double acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = 0.0;
    for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const double xe = x[e];
        double yv[G];
#pragma unroll
        for (int g = 0; g < G; ++g) yv[g] = yp[g][e];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = fma(xe, yv[g], acc[g]);
    }
    // the block reduction works on a power-of-two width (its slices must tile
    // the CTA): the G sums padded with zeros, of which only G are formed
    constexpr int GP = G <= 1 ? 1 : G <= 2 ? 2 : G <= 4 ? 4 : G <= 8 ? 8 : 16;
    double accp[GP];
#pragma unroll
    for (int g = 0; g < GP; ++g) accp[g] = g < G ? acc[g] : 0.0;
    const double tot = block_sums<GP, kKThreads>(accp, G, sh);
    if ((int)threadIdx.x < G) partial[(size_t)(v0 + threadIdx.x) * gridDim.x + blockIdx.x] = tot;
}

// partial[v * nchunk + chunk] = sum_{e in chunk} x[e] * Y_v[e], v < nv, and
// if want_xx, partial[nv * nchunk + chunk] = sum x[e]^2: groups of kDotGroup
// vectors, then one group of the remaining count
__device__ void chunk_dots(long e0, long e1, const double* __restrict__ x, const double* __restrict__ Y,
                           long ld, int nv, int want_xx, double* __restrict__ partial) {
    // sized for the widest reduction (kDotGroup): narrower ones need less
    __shared__ double sh[(kKThreads + kKThreads / kDotGroup) * (kDotGroup + 1)];
    const int tot = nv + want_xx;
    int v0 = 0;
    for (; v0 + kDotGroup <= tot; v0 += kDotGroup)
        chunk_dots_fixed<kDotGroup>(e0, e1, x, Y, ld, v0, want_xx && v0 + kDotGroup == tot, partial, sh);
    const bool xx = want_xx != 0;
    switch (tot - v0) {
#define REM(R) \
    case R: chunk_dots_fixed<R>(e0, e1, x, Y, ld, v0, xx, partial, sh); break;
        REM(1) REM(2) REM(3) REM(4) REM(5) REM(6) REM(7) REM(8) REM(9) REM(10) REM(11) REM(12) REM(13) REM(14)
        REM(15)
#undef REM
        default: break;
    }
}

// True in every thread of the CTA that finishes last; that CTA has seen the
// partials of every other CTA.  Resets the ticket for the next launch.
__device__ __forceinline__ bool last_cta(unsigned* ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
        if (last) *ticket = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// out[v] = sum of the chunk partials partial[v * nchunk + c], one warp per v;
// lane l sums chunks l, l+32, ... in four interleaved accumulators (their loads
// are independent), a fixed order for a fixed chunk count
__device__ __forceinline__ void finish_sums(int nv, const double* partial, double* out) {
    const int lane = threadIdx.x & 31;
    const int nchunk = gridDim.x;
    for (int v = threadIdx.x >> 5; v < nv; v += blockDim.x >> 5) {
        const double* p = partial + (size_t)v * nchunk;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int c = lane;
        for (; c + 96 < nchunk; c += 128) {
            s0 += __ldcg(p + c);
            s1 += __ldcg(p + c + 32);
            s2 += __ldcg(p + c + 64);
            s3 += __ldcg(p + c + 96);
        }
        for (; c < nchunk; c += 32) s0 += __ldcg(p + c);
        double s = (s0 + s1) + (s2 + s3);
        s = warp_sum(s);
        if (lane == 0) out[v] = s;
    }
}

// Arnoldi bookkeeping (one thread): column j of the Hessenberg matrix from
// h1 + h2 and ||w||, breakdown test, previous rotations, the new rotation,
// the residual estimate |g_{j+1}|.  scal = {h_{j+1,j}, |g_{j+1}|, breakdown,
// ||w|| before orthogonalising}.
__device__ void givens_update(const GivensArgs& a, double wsq) {
    const int j = a.j, m = a.m;
    double* H = a.H;
    const double wn0 = sqrt(__ldcg(a.h1 + j + 1));  // ||w||^2 before orthogonalising
    for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = __ldcg(a.h1 + i) + __ldcg(a.h2 + i);
    const double hn = sqrt(wsq);
    H[(size_t)(j + 1) * m + j] = hn;
    const int breakdown = !(hn > 1e-14 * wn0);
    for (int i = 0; i < j; ++i) {
        const double x0 = H[(size_t)i * m + j], x1 = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = a.cs[i] * x0 + a.sn[i] * x1;
        H[(size_t)(i + 1) * m + j] = -a.sn[i] * x0 + a.cs[i] * x1;
    }
    const double x0 = H[(size_t)j * m + j], x1 = H[(size_t)(j + 1) * m + j];
    const double d = sqrt(x0 * x0 + x1 * x1);
    if (d == 0.0) {
        a.cs[j] = 1.0;
        a.sn[j] = 0.0;
    } else {
        a.cs[j] = x0 / d;
        a.sn[j] = x1 / d;
    }
    H[(size_t)j * m + j] = d;
    H[(size_t)(j + 1) * m + j] = 0.0;
    a.g[j + 1] = -a.sn[j] * a.g[j];
    a.g[j] = a.cs[j] * a.g[j];
    a.scal[0] = hn;
    a.scal[1] = fabs(a.g[j + 1]);
    a.scal[2] = breakdown ? 1.0 : 0.0;
    a.scal[3] = wn0;
}

__global__ void __launch_bounds__(kKThreads) multi_dot_kernel(long N, const double* __restrict__ x,
                                                              const double* __restrict__ Y, long ld, int nv,
                                                              int want_xx, double* __restrict__ partial,
                                                              double* __restrict__ out, unsigned* ticket,
                                                              const unsigned* cond) {
    if (cond && __ldcg(cond) == 0u) return;  // a conditional pass that is not needed (every CTA)
    long e0, e1;
    chunk_range(N, &e0, &e1);
    chunk_dots(e0, e1, x, Y, ld, nv, want_xx, partial);
    if (last_cta(ticket)) finish_sums(nv + want_xx, partial, out);
}

// x -= sign * sum_v h[v] Y_v over the chunk, then (mode 1) the dots of the new
// x with Y_0..Y_{nv-1} into out, (mode 2) its squared norm into out (and the
// Givens update when do_givens), (mode 3) as 2, with the reorthogonalisation
// test of the Arnoldi step in the last CTA, (mode 0) nothing.  cond: the pass
// runs only where *cond is nonzero.
__global__ void __launch_bounds__(kKThreads) axpy_dot_kernel(long N, double* __restrict__ x,
                                                             const double* __restrict__ Y, long ld, int nv,
                                                             const double* __restrict__ h, double sign, int mode,
                                                             double* __restrict__ partial, double* __restrict__ out,
                                                             unsigned* ticket, GivensArgs ga, int do_givens,
                                                             const unsigned* cond, unsigned* reorth) {
    if (cond && __ldcg(cond) == 0u) return;
    __shared__ double sh_h[kMaxRestart + 1];
    for (int v = threadIdx.x; v < nv; v += blockDim.x) sh_h[v] = sign * h[v];
    __syncthreads();
    long e0, e1;
    chunk_range(N, &e0, &e1);
    // the basis vectors in groups of 8: the 8 loads are issued before the
    // dependent FMA chain (same order of the sum as one vector at a time)
    constexpr int kAxpyGroup = 8;
    for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        double t = x[e];
        int v = 0;
        for (; v + kAxpyGroup <= nv; v += kAxpyGroup) {
            double yv[kAxpyGroup];
#pragma unroll
            for (int g = 0; g < kAxpyGroup; ++g) yv[g] = Y[(size_t)(v + g) * ld + e];
#pragma unroll
            for (int g = 0; g < kAxpyGroup; ++g) t = fma(-sh_h[v + g], yv[g], t);
        }
        for (; v < nv; ++v) t = fma(-sh_h[v], Y[(size_t)v * ld + e], t);
        x[e] = t;
    }
    if (mode == 0) return;
    __syncthreads();
    if (mode == 1) chunk_dots(e0, e1, x, Y, ld, nv, 0, partial);
    else chunk_dots(e0, e1, x, Y, ld, 0, 1, partial);
    if (last_cta(ticket)) {
        finish_sums(mode == 1 ? nv : 1, partial, out);
        if (mode == 3) {
            // one projection is enough unless it removed nearly all of w
            // (||w1|| < eta ||w||, eta = 0.01); otherwise the step projects
            // again (the conditional passes) and its Givens update waits for it
            __syncthreads();
            if (threadIdx.x == 0) {
                const double w1 = __ldcg(out), w0 = __ldcg(ga.h1 + ga.j + 1);
                const unsigned need = !(w1 >= kReorthRatio * w0);
                *reorth = need;
                if (!need) {
                    double* h2 = const_cast<double*>(ga.h2);
                    for (int i = 0; i <= ga.j; ++i) h2[i] = 0.0;
                    givens_update(ga, w1);
                }
            }
        } else if (do_givens) {
            __syncthreads();
            if (threadIdx.x == 0) givens_update(ga, __ldcg(out));
        }
    }
}

int launch_multi_dot(long N, const double* x, const double* Y, long ld, int nv, int want_xx, double* partial,
                     double* out, unsigned* ticket, cudaStream_t s, const unsigned* cond) {
    multi_dot_kernel<<<krylov_chunks(N), kKThreads, 0, s>>>(N, x, Y, ld, nv, want_xx, partial, out, ticket, cond);
    return launched(1);
}
int launch_axpy_dot(long N, double* x, const double* Y, long ld, int nv, const double* h, double sign, int mode,
                    double* partial, double* out, unsigned* ticket, const GivensArgs* ga, cudaStream_t s,
                    const unsigned* cond, unsigned* reorth) {
    GivensArgs g{};
    if (ga) g = *ga;
    axpy_dot_kernel<<<krylov_chunks(N), kKThreads, 0, s>>>(N, x, Y, ld, nv, h, sign, mode, partial, out, ticket, g,
                                                           ga ? 1 : 0, cond, reorth);
    return launched(1);
}

// y = H(0:k, 0:k)^{-1} g(0:k), upper triangular
__global__ void solve_upper_kernel(int k, int m, const double* __restrict__ H, const double* __restrict__ g,
                                   double* __restrict__ y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int c = i + 1; c < k; ++c) s -= H[(size_t)i * m + c] * y[c];
        y[i] = s / H[(size_t)i * m + i];
    }
}

// y = x / scal[0] unless the breakdown flag scal[2] is set
__global__ void scale_kernel(long N, const double* __restrict__ x, const double* __restrict__ scal,
                             double* __restrict__ y, int check_breakdown) {
    if (check_breakdown && scal[2] != 0.0) return;
    // one division per thread and a product per element: an FP64 division
    // per element costs about ten FP64 operations, and GB300 issues two per
    // clock per SM (within an ulp of the quotient)
    const double rden = 1.0 / scal[0];
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long)gridDim.x * blockDim.x)
        y[e] = x[e] * rden;
}

// g = (beta, 0, ..., 0) with beta = sqrt(*bsq); scal[0] = beta
__global__ void init_g_kernel(int m, const double* __restrict__ bsq, double* __restrict__ g,
                              double* __restrict__ scal) {
    const int t = threadIdx.x;
    const double beta = sqrt(bsq[0]);
    for (int i = t; i <= m; i += blockDim.x) g[i] = (i == 0) ? beta : 0.0;
    if (t == 0) scal[0] = beta;
}

int launch_solve_upper(int k, int m, const double* H, const double* g, double* y, cudaStream_t s) {
    solve_upper_kernel<<<1, 32, 0, s>>>(k, m, H, g, y);
    return launched(1);
}
int launch_scale(long N, const double* x, const double* scal, double* y, int check_breakdown, cudaStream_t s) {
    long g = (N + 255) / 256;
    scale_kernel<<<(int)(g < 1216 ? (g > 0 ? g : 1) : 1216), 256, 0, s>>>(N, x, scal, y, check_breakdown);
    return launched(1);
}
int launch_init_g(int m, const double* bsq, double* g, double* scal, cudaStream_t s) {
    init_g_kernel<<<1, 64, 0, s>>>(m, bsq, g, scal);
    return launched(1);
}

}  // namespace bamg
