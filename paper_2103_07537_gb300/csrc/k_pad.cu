// Field blocks of unequal size (Algorithm 1 allows fields of any width): the
// system runs padded.  Every field is filled up to the widest field's fmax
// dofs with dummy dofs that carry one nonzero, on their own diagonal, and no
// coupling; the right-hand side and iterate are zero there.  Every step of
// the method then keeps the dummy entries at zero (residual, sub-solve with
// the block-diagonal inverse, restriction, Galerkin product, coarsest solve,
// Krylov vectors) and leaves the given dofs' values those of the unpadded
// method, so the padded system with equal fields computes it exactly (up to
// the order of rounding).
#include "common.cuh"

namespace bamg {

// one warp per block row i: the padded blocks of the row; the dummy dofs'
// diagonal entry is the largest magnitude in node i's given diagonal block
// (1 where that is zero), which keeps the padded matrix's scale.  The row
// range is clamped to the nnzb stored blocks: the pattern is validated by the
// setup that follows, so an invalid row_ptr reads nothing out of bounds here.
__global__ void __launch_bounds__(256) pad_values_kernel(PadMap pm, int n, int nnzb, const int* __restrict__ rp,
                                                         const int* __restrict__ ci,
                                                         const double* __restrict__ vals, double* __restrict__ vp) {
    const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    pdl_wait();
    if (w >= n) return;
    const int i = (int)w;
    const int k0 = min(max(rp[i], 0), nnzb), k1 = min(max(rp[i + 1], k0), nnzb);
    const int b = pm.b, bp = pm.bp, bb = b * b, bpp = bp * bp;
    double dmax = 0.0;
    for (int k = k0; k < k1; ++k)
        if (ci[k] == i)
            for (int e = lane; e < bb; e += 32) dmax = fmax(dmax, fabs(vals[(size_t)k * bb + e]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (!(dmax > 0.0) || !isfinite(dmax)) dmax = 1.0;
    for (int k = k0; k < k1; ++k) {
        const bool diag = ci[k] == i;
        for (int e = lane; e < bpp; e += 32) {
            const int r = e / bp, c = e - r * bp;
            const int sr = pm.src[r], sc = pm.src[c];
            double v = 0.0;
            if (sr >= 0 && sc >= 0) v = vals[(size_t)k * bb + sr * b + sc];
            else if (diag && r == c) v = dmax;
            vp[(size_t)k * bpp + e] = v;
        }
    }
}

int launch_pad_values(const PadMap& pm, int n, int nnzb, const int* rp, const int* ci, const double* vals,
                      double* vp, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    if (launch_k(pad_values_kernel, ceil_div((long)n * 32, 256), 256, 0, s, pm, n, nnzb, rp, ci, vals, vp) !=
        cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}

// xp (n x bp) from x (n x b): zero at the dummy dofs
__global__ void pad_vec_kernel(PadMap pm, long n, const double* __restrict__ x, double* __restrict__ xp) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    pdl_wait();
    if (e >= n * pm.bp) return;
    const long i = e / pm.bp;
    const int q = (int)(e - i * pm.bp);
    const int d = pm.src[q];
    xp[e] = d >= 0 ? x[i * pm.b + d] : 0.0;
}

// x (n x b) from xp (n x bp): the given dofs
__global__ void unpad_vec_kernel(PadMap pm, long n, const double* __restrict__ xp, double* __restrict__ x) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    pdl_wait();
    if (e >= n * pm.b) return;
    const long i = e / pm.b;
    const int d = (int)(e - i * pm.b);
    x[e] = xp[i * pm.bp + pm.dst[d]];
}

int launch_pad_vec(const PadMap& pm, long n, const double* x, double* xp, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    if (launch_k(pad_vec_kernel, ceil_div(n * pm.bp, 256), 256, 0, s, pm, n, x, xp) != cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}

int launch_unpad_vec(const PadMap& pm, long n, const double* xp, double* x, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    if (launch_k(unpad_vec_kernel, ceil_div(n * pm.b, 256), 256, 0, s, pm, n, xp, x) != cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}

}  // namespace bamg
