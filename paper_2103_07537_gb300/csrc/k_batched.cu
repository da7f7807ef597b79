// Kernels for a batch of independent systems solved together (one block-
// diagonal operator): per-system (segmented) reductions and updates of the
// outer FGMRES, per-system Arnoldi bookkeeping, and the per-system dense LU,
// inverse and GEMV of the coarsest level.
//
// Vectors are the concatenation of the systems' vectors; a fixed table cuts
// every system into chunks (one CTA each) so that all sums are deterministic:
// chunk partials are reduced in a fixed tree, then added in chunk order per
// system.
#include <math.h>

#include "common.cuh"

namespace bamg {

constexpr int kBThreads = 256;
constexpr int kBGroup = 16;

// partial[v * nchunk + c] = sum over chunk c of x . Y_v (v < nv), and x . x
// at v = nv when want_xx; CTA per chunk
__device__ void seg_chunk_dots(long e0, long e1, const double* __restrict__ x, const double* __restrict__ Y,
                               long ld, int nv, int want_xx, double* __restrict__ partial, int c, int nchunk) {
    __shared__ double sh[(kBThreads + kBThreads / kBGroup) * (kBGroup + 1)];
    for (int v0 = 0; v0 < nv + want_xx; v0 += kBGroup) {
        double acc[kBGroup];
#pragma unroll
        for (int g = 0; g < kBGroup; ++g) acc[g] = 0.0;
        for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const double xe = x[e];
#pragma unroll
            for (int g = 0; g < kBGroup; ++g) {
                const int v = v0 + g;
                if (v < nv) acc[g] = fma(xe, Y[(size_t)v * ld + e], acc[g]);
                else if (v == nv && want_xx) acc[g] = fma(xe, xe, acc[g]);
            }
        }
        const int gn = min(kBGroup, nv + want_xx - v0);
        const double tot = block_sums<kBGroup, kBThreads>(acc, gn, sh);
        if ((int)threadIdx.x < gn) partial[(size_t)(v0 + threadIdx.x) * nchunk + c] = tot;
    }
}

__global__ void __launch_bounds__(kBThreads) seg_dots_kernel(SegTable t, const double* __restrict__ x,
                                                             const double* __restrict__ Y, long ld, int nv,
                                                             int want_xx, double* __restrict__ partial) {
    const int c = blockIdx.x;
    seg_chunk_dots(t.chunk_e0[c], t.chunk_e1[c], x, Y, ld, nv, want_xx, partial, c, t.nchunk);
}

// x -= sign * sum_v h_s[v] Y_v on the chunks of active systems (h_s = h + s * ldh),
// then mode 1: dots with Y_v, mode 2: x . x, mode 0: nothing.  Chunks of inactive
// systems write zero partials.
__global__ void __launch_bounds__(kBThreads) seg_axpy_dots_kernel(SegTable t, double* __restrict__ x,
                                                                  const double* __restrict__ Y, long ld, int nv,
                                                                  const double* __restrict__ h, int ldh, double sign,
                                                                  int mode, const int* __restrict__ active,
                                                                  double* __restrict__ partial) {
    __shared__ double sh_h[kMaxRestart + 1];
    const int c = blockIdx.x;
    const int s = t.chunk_sys[c];
    const long e0 = t.chunk_e0[c], e1 = t.chunk_e1[c];
    const bool on = active == nullptr || active[s] != 0;
    if (on) {
        for (int v = threadIdx.x; v < nv; v += blockDim.x) sh_h[v] = sign * h[(size_t)s * ldh + v];
        __syncthreads();
        for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            double tt = x[e];
            for (int v = 0; v < nv; ++v) tt = fma(-sh_h[v], Y[(size_t)v * ld + e], tt);
            x[e] = tt;
        }
        __syncthreads();
    }
    if (mode == 0) return;
    const int nout = mode == 1 ? nv : 1;
    if (!on) {
        for (int v = threadIdx.x; v < nout; v += blockDim.x) partial[(size_t)v * t.nchunk + c] = 0.0;
        return;
    }
    if (mode == 1) seg_chunk_dots(e0, e1, x, Y, ld, nv, 0, partial, c, t.nchunk);
    else seg_chunk_dots(e0, e1, x, Y, ld, 0, 1, partial, c, t.nchunk);
}

// out[s * ldo + v] = sum over the chunks of system s (in order) of partial[v][c]
__global__ void seg_finish_kernel(SegTable t, int nv, const double* __restrict__ partial, double* __restrict__ out,
                                  int ldo) {
    const int s = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int c0 = t.sys_chunk[s], c1 = t.sys_chunk[s + 1];
    for (int v = threadIdx.x >> 5; v < nv; v += blockDim.x >> 5) {
        double acc = 0.0;
        for (int c = c0 + lane; c < c1; c += 32) acc += partial[(size_t)v * t.nchunk + c];
        acc = warp_sum(acc);
        if (lane == 0) out[(size_t)s * ldo + v] = acc;
    }
}

// Arnoldi bookkeeping of step j for every system in the cycle (thread per
// system); per-system arrays are strided by the restart length.
__global__ void seg_givens_kernel(int nsys, int j, int m, const double* __restrict__ h1,
                                  const double* __restrict__ h2, const double* __restrict__ wsq,
                                  double* __restrict__ Hb, double* __restrict__ csb, double* __restrict__ snb,
                                  double* __restrict__ gb, double* __restrict__ scalb, const int* __restrict__ incycle) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || !incycle[s]) return;
    const double* a1 = h1 + (size_t)s * (m + 2);
    const double* a2 = h2 + (size_t)s * (m + 2);
    double* H = Hb + (size_t)s * (m + 1) * m;
    double* cs = csb + (size_t)s * m;
    double* sn = snb + (size_t)s * m;
    double* g = gb + (size_t)s * (m + 1);
    double* scal = scalb + (size_t)s * 4;
    const double wn0 = sqrt(a1[j + 1]);
    for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = a1[i] + a2[i];
    const double hn = sqrt(wsq[s]);
    H[(size_t)(j + 1) * m + j] = hn;
    const int breakdown = !(hn > 1e-14 * wn0);
    for (int i = 0; i < j; ++i) {
        const double x0 = H[(size_t)i * m + j], x1 = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * x0 + sn[i] * x1;
        H[(size_t)(i + 1) * m + j] = -sn[i] * x0 + cs[i] * x1;
    }
    const double x0 = H[(size_t)j * m + j], x1 = H[(size_t)(j + 1) * m + j];
    const double d = sqrt(x0 * x0 + x1 * x1);
    if (d == 0.0) {
        cs[j] = 1.0;
        sn[j] = 0.0;
    } else {
        cs[j] = x0 / d;
        sn[j] = x1 / d;
    }
    H[(size_t)j * m + j] = d;
    H[(size_t)(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    scal[0] = hn;
    scal[1] = fabs(g[j + 1]);
    scal[2] = breakdown ? 1.0 : 0.0;
    scal[3] = wn0;
}

// y_out = x / scal_s[0] on the chunks of systems in the cycle without breakdown
// (check_breakdown) or of active systems (initial normalisation)
__global__ void __launch_bounds__(kBThreads) seg_scale_kernel(SegTable t, const double* __restrict__ x,
                                                              const double* __restrict__ scalb,
                                                              double* __restrict__ y, const int* __restrict__ on,
                                                              int check_breakdown) {
    const int c = blockIdx.x;
    const int s = t.chunk_sys[c];
    if (!on[s]) return;
    const double* scal = scalb + (size_t)s * 4;
    if (check_breakdown && scal[2] != 0.0) return;
    const double rden = 1.0 / scal[0];  // a product per element (an FP64 division costs ~10 FP64 operations)
    for (long e = t.chunk_e0[c] + threadIdx.x; e < t.chunk_e1[c]; e += blockDim.x) y[e] = x[e] * rden;
}

// g_s = (beta_s, 0, ...), scal_s[0] = beta_s = sqrt(bsq_s)
__global__ void seg_init_g_kernel(int nsys, int m, const double* __restrict__ bsq, double* __restrict__ gb,
                                  double* __restrict__ scalb) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const double beta = sqrt(bsq[s]);
    for (int i = 0; i <= m; ++i) gb[(size_t)s * (m + 1) + i] = i == 0 ? beta : 0.0;
    scalb[(size_t)s * 4] = beta;
}

// y_s = H_s(0:k_s, 0:k_s)^{-1} g_s(0:k_s), zero beyond k_s
__global__ void seg_solve_upper_kernel(int nsys, int m, const int* __restrict__ kk, const double* __restrict__ Hb,
                                       const double* __restrict__ gb, double* __restrict__ yb) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const int k = kk[s];
    const double* H = Hb + (size_t)s * (m + 1) * m;
    const double* g = gb + (size_t)s * (m + 1);
    double* y = yb + (size_t)s * m;
    for (int i = k; i < m; ++i) y[i] = 0.0;
    for (int i = k - 1; i >= 0; --i) {
        double acc = g[i];
        for (int c = i + 1; c < k; ++c) acc -= H[(size_t)i * m + c] * y[c];
        y[i] = acc / H[(size_t)i * m + i];
    }
}

int launch_seg_dots(const SegTable& t, const double* x, const double* Y, long ld, int nv, int want_xx,
                    double* partial, double* out, int ldo, cudaStream_t s) {
    seg_dots_kernel<<<t.nchunk, kBThreads, 0, s>>>(t, x, Y, ld, nv, want_xx, partial);
    seg_finish_kernel<<<t.nsys, 256, 0, s>>>(t, nv + want_xx, partial, out, ldo);
    return launched(2);
}
int launch_seg_axpy_dots(const SegTable& t, double* x, const double* Y, long ld, int nv, const double* h, int ldh,
                         double sign, int mode, const int* active, double* partial, double* out, int ldo,
                         cudaStream_t s) {
    seg_axpy_dots_kernel<<<t.nchunk, kBThreads, 0, s>>>(t, x, Y, ld, nv, h, ldh, sign, mode, active, partial);
    if (mode == 0) return launched(1);
    seg_finish_kernel<<<t.nsys, 256, 0, s>>>(t, mode == 1 ? nv : 1, partial, out, ldo);
    return launched(2);
}
int launch_seg_givens(int nsys, int j, int m, const double* h1, const double* h2, const double* wsq, double* H,
                      double* cs, double* sn, double* g, double* scal, const int* incycle, cudaStream_t s) {
    seg_givens_kernel<<<ceil_div(nsys, 128), 128, 0, s>>>(nsys, j, m, h1, h2, wsq, H, cs, sn, g, scal, incycle);
    return launched(1);
}
int launch_seg_scale(const SegTable& t, const double* x, const double* scal, double* y, const int* on,
                     int check_breakdown, cudaStream_t s) {
    seg_scale_kernel<<<t.nchunk, kBThreads, 0, s>>>(t, x, scal, y, on, check_breakdown);
    return launched(1);
}
int launch_seg_init_g(int nsys, int m, const double* bsq, double* g, double* scal, cudaStream_t s) {
    seg_init_g_kernel<<<ceil_div(nsys, 128), 128, 0, s>>>(nsys, m, bsq, g, scal);
    return launched(1);
}
int launch_seg_solve_upper(int nsys, int m, const int* k, const double* H, const double* g, double* y,
                           cudaStream_t s) {
    seg_solve_upper_kernel<<<ceil_div(nsys, 128), 128, 0, s>>>(nsys, m, k, H, g, y);
    return launched(1);
}

// ---------------------------------------------------------------------------
// coarsest level of a batch: one dense block per system
// ---------------------------------------------------------------------------
// CTA per system: dense copy of its coarse rows (nodes off..off+nn-1), LU with
// partial pivoting (first maximum wins; rounded product then rounded
// difference), then the inverse column by column (thread per column) into
// inv + inv_off[s].  The factorisation lives in shared memory when it fits,
// else in the global work area work + inv_off[s].  piv and col: nd_total
// entries each, system s at node_off[s] * b.
constexpr int kBatchLuThreads = 256;
__global__ void __launch_bounds__(kBatchLuThreads) batched_lu_inverse_kernel(
    int b, const int* __restrict__ node_off, const long* __restrict__ inv_off, const int* __restrict__ rp,
    const int* __restrict__ ci, const double* __restrict__ vals, double* __restrict__ work, double* __restrict__ inv,
    int* __restrict__ piv_all, double* __restrict__ col_all, int smem_max_nd, int* err) {
    extern __shared__ double sm[];
    __shared__ double red_v[kBatchLuThreads / 32];
    __shared__ int red_i[kBatchLuThreads / 32];
    const int s = blockIdx.x;
    const int n0 = node_off[s], nn = node_off[s + 1] - n0;
    const int nd = nn * b;
    if (nd == 0) return;
    double* a = nd <= smem_max_nd ? sm : work + inv_off[s];
    double* col = col_all + (size_t)n0 * b;
    int* piv = piv_all + (size_t)n0 * b;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int e = tid; e < nd * nd; e += blockDim.x) a[e] = 0.0;
    __syncthreads();
    for (int i = 0; i < nn; ++i)
        for (int k = rp[n0 + i]; k < rp[n0 + i + 1]; ++k) {
            const int j = ci[k] - n0;
            for (int e = tid; e < b * b; e += blockDim.x) {
                const int r = e / b, c = e - r * b;
                a[(size_t)(i * b + r) * nd + j * b + c] = vals[(size_t)k * b * b + e];
            }
        }
    __syncthreads();
    // infinity norm
    double m = 0.0;
    for (int r = tid; r < nd; r += blockDim.x) {
        double sum = 0.0;
        for (int c = 0; c < nd; ++c) sum += fabs(a[(size_t)r * nd + c]);
        m = fmax(m, sum);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red_v[wid] = m;
    __syncthreads();
    double norm = 0.0;
    for (int w = 0; w < kBatchLuThreads / 32; ++w) norm = fmax(norm, red_v[w]);
    __syncthreads();
    bool singular = norm == 0.0;
    for (int k = 0; k < nd; ++k) {
        double best = -1.0;
        int bi = nd;
        for (int r = k + tid; r < nd; r += blockDim.x) {
            const double v = fabs(a[(size_t)r * nd + k]);
            if (v > best) {
                best = v;
                bi = r;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            red_v[wid] = best;
            red_i[wid] = bi;
        }
        __syncthreads();
        double bv = red_v[0];
        int p = red_i[0];
        for (int w = 1; w < kBatchLuThreads / 32; ++w)
            if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < p)) {
                bv = red_v[w];
                p = red_i[w];
            }
        __syncthreads();
        if (!(bv >= 1e-14 * norm)) singular = true;
        if (tid == 0) piv[k] = p;
        if (p != k)
            for (int c = tid; c < nd; c += blockDim.x) {
                const double t = a[(size_t)k * nd + c];
                a[(size_t)k * nd + c] = a[(size_t)p * nd + c];
                a[(size_t)p * nd + c] = t;
            }
        __syncthreads();
        const double akk = a[(size_t)k * nd + k];
        for (int r = k + 1 + tid; r < nd; r += blockDim.x) col[r] = __ddiv_rn(a[(size_t)r * nd + k], akk);
        __syncthreads();
        const int mm = nd - k - 1;
        for (int e = tid; e < mm * mm; e += blockDim.x) {
            const int r = k + 1 + e / mm, c = k + 1 + e % mm;
            a[(size_t)r * nd + c] = __dsub_rn(a[(size_t)r * nd + c], __dmul_rn(col[r], a[(size_t)k * nd + c]));
        }
        for (int r = k + 1 + tid; r < nd; r += blockDim.x) a[(size_t)r * nd + k] = col[r];
        __syncthreads();
    }
    if (singular) {
        if (tid == 0) set_error(err, kDevSingularCoarse);
        return;
    }
    double* out = inv + inv_off[s];
    for (int c = tid; c < nd; c += blockDim.x) {
        int pos = c;  // P e_c: the row swaps applied in order to the unit vector
        for (int k = 0; k < nd; ++k) {
            const int pk = piv[k];
            if (pk == pos) pos = k;
            else if (k == pos) pos = pk;
        }
        // forward (unit lower) and backward substitution for column c, in out[:, c]
        for (int r = 0; r < nd; ++r) out[(size_t)r * nd + c] = 0.0;
        out[(size_t)pos * nd + c] = 1.0;
        for (int r = pos + 1; r < nd; ++r) {
            double acc = out[(size_t)r * nd + c];
            for (int k = pos; k < r; ++k) acc -= a[(size_t)r * nd + k] * out[(size_t)k * nd + c];
            out[(size_t)r * nd + c] = acc;
        }
        for (int r = nd - 1; r >= 0; --r) {
            double acc = out[(size_t)r * nd + c];
            for (int k = r + 1; k < nd; ++k) acc -= a[(size_t)r * nd + k] * out[(size_t)k * nd + c];
            out[(size_t)r * nd + c] = acc / a[(size_t)r * nd + r];
        }
    }
}

int batched_lu_inverse(int nsys, int b, int max_nd, const int* node_off, const long* inv_off, const int* rp,
                       const int* ci, const double* vals, double* work, double* inv, int* piv, double* col, int* err,
                       cudaStream_t s) {
    const int smem_max_nd = 156;  // nd^2 doubles <= 195 KB of shared memory
    const int use_nd = max_nd <= smem_max_nd ? max_nd : 0;
    const size_t smem = sizeof(double) * ((size_t)use_nd * use_nd + 1);
    BAMG_CUDA_TRY(cudaFuncSetAttribute(batched_lu_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(smem < 48 * 1024 ? 48 * 1024 : smem)));
    batched_lu_inverse_kernel<<<nsys, kBatchLuThreads, smem, s>>>(b, node_off, inv_off, rp, ci, vals, work, inv, piv,
                                                                  col, use_nd, err);
    return launched(1);
}

// y_r = sum_c Ainv_s[r - o_s][c] x_{o_s + c}: warp per coarse unknown r of system s
template <typename T>
__global__ void batched_gemv_kernel(int nd_total, int b, const int* __restrict__ row_sys,
                                    const int* __restrict__ node_off, const long* __restrict__ inv_off,
                                    const double* __restrict__ inv, const T* __restrict__ x, T* __restrict__ y) {
    pdl_wait();
    pdl_trigger();
    const int r = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= nd_total) return;
    const int s = row_sys[r];
    const int o = node_off[s] * b, nd = (node_off[s + 1] - node_off[s]) * b;
    const double* a = inv + inv_off[s] + (size_t)(r - o) * nd;
    double acc = 0.0;
    for (int c = lane; c < nd; c += 32) acc = fma(__ldg(a + c), (double)x[o + c], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[r] = (T)acc;
}

template <typename T>
int launch_batched_gemv(int nd_total, int b, const int* row_sys, const int* node_off, const long* inv_off,
                        const double* inv, const T* x, T* y, cudaStream_t s) {
    if (nd_total <= 0) return BAMG_OK;
    if (launch_k(batched_gemv_kernel<T>, ceil_div((long)nd_total * 32, 256), 256, 0, s, nd_total, b, row_sys, node_off,
                 inv_off, inv, x, y) != cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}
template int launch_batched_gemv<double>(int, int, const int*, const int*, const long*, const double*,
                                         const double*, double*, cudaStream_t);
template int launch_batched_gemv<float>(int, int, const int*, const int*, const long*, const double*, const float*,
                                        float*, cudaStream_t);

// every stored block stays inside its system's node range
__global__ void check_batch_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                   const int* __restrict__ node_sys, const int* __restrict__ node_off, int* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = node_sys[i];
    const int lo = node_off[s], hi = node_off[s + 1];
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] < lo || ci[k] >= hi) set_error(err, kDevBadPattern);
}

// node_sys[i] = s for node_off[s] <= i < node_off[s+1]
__global__ void fill_sys_kernel(int nsys, const int* __restrict__ node_off, int scale, int* __restrict__ out) {
    const int s = blockIdx.x;
    for (int i = node_off[s] * scale + threadIdx.x; i < node_off[s + 1] * scale; i += blockDim.x) out[i] = s;
}

int launch_check_batch(int n, const int* rp, const int* ci, const int* node_sys, const int* node_off, int* err,
                       cudaStream_t s) {
    check_batch_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, ci, node_sys, node_off, err);
    return launched(1);
}
int launch_fill_sys(int nsys, const int* node_off, int scale, int* out, cudaStream_t s) {
    fill_sys_kernel<<<nsys, 256, 0, s>>>(nsys, node_off, scale, out);
    return launched(1);
}

// coarse offsets: off_c[s] = rootid[off[s]] (the rank of the first root at or after the system start)
__global__ void coarse_offsets_kernel(int nsys, const int* __restrict__ off, const int* __restrict__ rank,
                                      int* __restrict__ off_c) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s <= nsys) off_c[s] = rank[off[s]];
}
int launch_coarse_offsets(int nsys, const int* off, const int* rank, int* off_c, cudaStream_t s) {
    coarse_offsets_kernel<<<ceil_div(nsys + 1, 128), 128, 0, s>>>(nsys, off, rank, off_c);
    return launched(1);
}

}  // namespace bamg
