// Schwarz sub-solve of Algorithm 1 (Sec. 5: one additive Schwarz iteration
// with overlap one approximates each A_ff^{-1} in the paper's runs), in the
// restricted form: every node takes the local solution of its own subdomain.
//
// Subdomains are the level's aggregates (of one node field, with node
// fields), each extended by `overlap` layers of neighbours in the graph of
// A_ff (neighbours in the same node field), nodes ascending; one subdomain
// per aggregate and field block.  A_I is the field-f sub-block matrix
// between the subdomain's nodes.  Setup factors A_I in FP64 by LU with
// partial pivoting (first maximum wins, as the coarsest solve) and keeps only
// the rows of A_I^{-1} that belong to the aggregate's own nodes (the
// restricted form never uses the others): X_I, own_rows x m, stored column by
// column so that the cycle reads it coalesced.  A field step is then
//   r_f = rhs_f - A_{f,*} x_in                (one thread per scalar row)
//   x~_i = X_I r_f|_I for the own nodes i of every aggregate I (one warp per
//   subdomain: gather r over the subdomain, then lanes = own rows)
//   x_f += omega x~_f
// with no dependence between subdomains, so one launch of each per field step.
#include "common.cuh"
#include "bgs_body.cuh"

namespace bamg {

constexpr int kSdMaxM = 160;  // unknowns of one subdomain (nodes x fb)

// the subdomain of aggregate I: members, then `overlap` layers of neighbours
// of the same node field, ascending; returns the count (or -1 above kSdMaxM
// nodes); list may be null (count only)
__device__ int subdomain_nodes(int I, const int* __restrict__ agg_ptr, const int* __restrict__ members,
                               const int* __restrict__ rp, const int* __restrict__ ci,
                               const int* __restrict__ node_field, int overlap, int* buf) {
    int cnt = 0;
    for (int t = agg_ptr[I]; t < agg_ptr[I + 1]; ++t) {
        if (cnt == kSdMaxM) return -1;
        buf[cnt++] = members[t];
    }
    for (int layer = 0; layer < overlap; ++layer) {
        const int c0 = cnt;
        for (int t = 0; t < c0; ++t) {
            const int i = buf[t];
            for (int k = rp[i]; k < rp[i + 1]; ++k) {
                const int j = ci[k];
                if (node_field && node_field[j] != node_field[i]) continue;
                bool seen = false;
                for (int u = 0; u < cnt && !seen; ++u) seen = buf[u] == j;
                if (seen) continue;
                if (cnt == kSdMaxM) return -1;
                buf[cnt++] = j;
            }
        }
    }
    // ascending (insertion sort; at most kSdMaxM entries)
    for (int t = 1; t < cnt; ++t) {
        const int v = buf[t];
        int u = t;
        while (u > 0 && buf[u - 1] > v) {
            buf[u] = buf[u - 1];
            --u;
        }
        buf[u] = v;
    }
    return cnt;
}

__global__ void sd_count_kernel(int n_agg, const int* __restrict__ agg_ptr, const int* __restrict__ members,
                                const int* __restrict__ rp, const int* __restrict__ ci,
                                const int* __restrict__ node_field, int overlap, int* __restrict__ cnt) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n_agg) return;
    int buf[kSdMaxM];
    cnt[I] = subdomain_nodes(I, agg_ptr, members, rp, ci, node_field, overlap, buf);
}

__global__ void sd_fill_kernel(int n_agg, const int* __restrict__ agg_ptr, const int* __restrict__ members,
                               const int* __restrict__ rp, const int* __restrict__ ci,
                               const int* __restrict__ node_field, int overlap, const int* __restrict__ sd_ptr,
                               int* __restrict__ sd_nodes) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n_agg) return;
    int buf[kSdMaxM];
    const int cnt = subdomain_nodes(I, agg_ptr, members, rp, ci, node_field, overlap, buf);
    for (int t = 0; t < cnt; ++t) sd_nodes[sd_ptr[I] + t] = buf[t];
}

// One CTA per (aggregate I, field f): A_I in shared memory, its LU with
// partial pivoting, then the own rows of A_I^{-1}: with P A = L U,
// e_p^T A^{-1} = (U^{-T} e_p)^T L^{-1} P, i.e. U^T w = e_p (forward),
// L^T v = w (backward, unit diagonal), row = P^T v (the swaps undone in
// reverse order).  One thread per own row; w / v in a per-thread array.
__global__ void __launch_bounds__(128) sd_factor_kernel(int F, int b, int fb, const int* __restrict__ sd_ptr,
                                                        const int* __restrict__ sd_nodes,
                                                        const int* __restrict__ agg_ptr,
                                                        const int* __restrict__ members, const int* __restrict__ rp,
                                                        const int* __restrict__ ci, const double* __restrict__ vals,
                                                        const long* __restrict__ x_off, double* __restrict__ X,
                                                        int* err) {
    extern __shared__ double sa[];  // m * m
    __shared__ int piv[kSdMaxM];
    __shared__ double s_norm;
    __shared__ double s_bv[128];
    __shared__ int s_bi[128];
    const int q = blockIdx.x;
    const int I = q / F, f = q - I * F;
    const int s0 = sd_ptr[I], cnt = sd_ptr[I + 1] - s0, m = cnt * fb;
    const int f0 = f * fb;
    const int tid = threadIdx.x, nt = blockDim.x;
    const size_t bb = (size_t)b * b;
    for (int e = tid; e < m * m; e += nt) sa[e] = 0.0;
    __syncthreads();
    // A_I: row p of the subdomain, columns found by binary search in the list
    for (int p = tid; p < cnt; p += nt) {
        const int i = sd_nodes[s0 + p];
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            int lo = 0, hi = cnt;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sd_nodes[s0 + mid] < j) lo = mid + 1;
                else hi = mid;
            }
            if (lo == cnt || sd_nodes[s0 + lo] != j) continue;
            for (int r = 0; r < fb; ++r)
                for (int c = 0; c < fb; ++c)
                    sa[(size_t)(p * fb + r) * m + lo * fb + c] = vals[(size_t)k * bb + (f0 + r) * b + f0 + c];
        }
    }
    __syncthreads();
    if (tid == 0) {  // infinity norm for the singularity test
        double nrm = 0.0;
        for (int r = 0; r < m; ++r) {
            double sr = 0.0;
            for (int c = 0; c < m; ++c) sr += fabs(sa[(size_t)r * m + c]);
            if (sr > nrm) nrm = sr;
        }
        s_norm = nrm;
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        // pivot: the first row of maximum |a_rk|, r >= k
        double bv = -1.0;
        int bi = k;
        for (int r = k + tid; r < m; r += nt) {
            const double v = fabs(sa[(size_t)r * m + k]);
            if (v > bv) {
                bv = v;
                bi = r;
            }
        }
        s_bv[tid] = bv;
        s_bi[tid] = bi;
        __syncthreads();
        if (tid == 0) {
            double best = s_bv[0];
            int bestr = s_bi[0];
            for (int t = 1; t < nt; ++t)
                if (s_bv[t] > best || (s_bv[t] == best && s_bi[t] < bestr)) {
                    best = s_bv[t];
                    bestr = s_bi[t];
                }
            if (!(best >= 1e-14 * s_norm) || s_norm == 0.0) set_error(err, kDevSingularBlock);
            piv[k] = bestr;
        }
        __syncthreads();
        const int p = piv[k];
        if (p != k)
            for (int c = tid; c < m; c += nt) {
                const double t = sa[(size_t)k * m + c];
                sa[(size_t)k * m + c] = sa[(size_t)p * m + c];
                sa[(size_t)p * m + c] = t;
            }
        __syncthreads();
        const double akk = sa[(size_t)k * m + k];
        for (int r = k + 1 + tid; r < m; r += nt) {
            const double l = akk != 0.0 ? __ddiv_rn(sa[(size_t)r * m + k], akk) : 0.0;
            sa[(size_t)r * m + k] = l;
            for (int c = k + 1; c < m; ++c)
                sa[(size_t)r * m + c] = __dsub_rn(sa[(size_t)r * m + c], __dmul_rn(l, sa[(size_t)k * m + c]));
        }
        __syncthreads();
    }
    // own rows: members of I (ascending, a subset of the ascending list)
    const int own = (agg_ptr[I + 1] - agg_ptr[I]) * fb;
    double* Xq = X + x_off[q];
    for (int t = tid; t < own; t += nt) {
        const int node = members[agg_ptr[I] + t / fb];
        int lo = 0, hi = cnt;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sd_nodes[s0 + mid] < node) lo = mid + 1;
            else hi = mid;
        }
        const int prow = lo * fb + t % fb;
        double w[kSdMaxM];
        for (int k = 0; k < m; ++k) {  // U^T w = e_prow
            double s = k == prow ? 1.0 : 0.0;
            for (int j = 0; j < k; ++j) s -= sa[(size_t)j * m + k] * w[j];
            w[k] = s / sa[(size_t)k * m + k];
        }
        for (int k = m - 1; k >= 0; --k) {  // L^T v = w, in place
            double s = w[k];
            for (int j = k + 1; j < m; ++j) s -= sa[(size_t)j * m + k] * w[j];
            w[k] = s;
        }
        for (int k = m - 1; k >= 0; --k) {  // P^T v
            const int pk = piv[k];
            const double tmp = w[k];
            w[k] = w[pk];
            w[pk] = tmp;
        }
        for (int c = 0; c < m; ++c) Xq[(size_t)c * own + t] = w[c];
    }
}

int schwarz_setup_count(int n_agg, const int* agg_ptr, const int* members, const int* rp, const int* ci,
                        const int* node_field, int overlap, int* cnt, cudaStream_t s) {
    if (n_agg <= 0) return BAMG_OK;
    sd_count_kernel<<<ceil_div(n_agg, 64), 64, 0, s>>>(n_agg, agg_ptr, members, rp, ci, node_field, overlap, cnt);
    return launched(1);
}

int schwarz_setup_fill(int n_agg, int F, int b, int fb, int max_m, const int* agg_ptr, const int* members,
                       const int* rp, const int* ci, const int* node_field, int overlap, const int* sd_ptr,
                       int* sd_nodes, const double* vals, const long* x_off, double* X, int* err, cudaStream_t s) {
    if (n_agg <= 0) return BAMG_OK;
    if (max_m > kSdMaxM) return BAMG_EUNSUPPORTED;
    sd_fill_kernel<<<ceil_div(n_agg, 64), 64, 0, s>>>(n_agg, agg_ptr, members, rp, ci, node_field, overlap, sd_ptr,
                                                       sd_nodes);
    const size_t smem = (size_t)max_m * max_m * sizeof(double);
    BAMG_CUDA_TRY(cudaFuncSetAttribute(sd_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    sd_factor_kernel<<<n_agg * F, 128, smem, s>>>(F, b, fb, sd_ptr, sd_nodes, agg_ptr, members, rp, ci, vals, x_off,
                                                  X, err);
    return launched(2);
}

// ---------------------------------------------------------------------------
// cycle kernels
// ---------------------------------------------------------------------------
// rf[i][r] = rhs[i][f0 + r] - sum_j A[i,j](f0 + r, :) (x_in + P uc)_j, one
// thread per scalar row of the field (x_in null: rf = rhs_f)
template <typename T, int B, int FB, bool FM>
__global__ void __launch_bounds__(256) field_residual_kernel(int n, int field, const int* __restrict__ rp,
                                                             const int* __restrict__ ci, const T* __restrict__ vals,
                                                             const T* __restrict__ x_in, const T* __restrict__ uc,
                                                             const int* __restrict__ agg, const T* __restrict__ rhs,
                                                             T* __restrict__ rf) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / FB);
    if (i >= n) return;
    const int r = (int)(t - (long)i * FB);
    const int f0 = field * FB;
    pdl_wait();
    pdl_trigger();
    T acc = T(0);
    if (x_in) {
        const int k0 = __ldg(rp + i), k1 = __ldg(rp + i + 1);
        const T* vb = vrow<T, B, FB, FM>(vals, k0, k1, k0, f0 + r);
        constexpr int VS = vstride<T, B, FB, FM>();
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            const int j = __ldg(ci + k);
            T a[B], xv[B];
            load_row<T, B>(vb + (size_t)(k - k0) * VS, a);
            load_row<T, B>(x_in + (size_t)j * B, xv);
            if (uc) {
                T pv[B];
                load_row<T, B>(uc + (size_t)__ldg(agg + j) * B, pv);
#pragma unroll
                for (int c = 0; c < B; ++c) xv[c] += pv[c];
            }
#pragma unroll
            for (int c = 0; c < B; ++c) acc = fma(a[c], xv[c], acc);
        }
    }
    rf[(size_t)i * FB + r] = rhs[(size_t)i * B + f0 + r] - acc;
}

// one warp per subdomain (aggregate I0 + w of the field step): r over the
// subdomain into shared memory, then lane t of each pass of 32 own rows
// x~ = X_I[:, t] . r_I, and x_out of the own node = x_in (+ P uc), field f
// += omega x~ (the lane of own row (node, c) also copies component c of the
// other fields)
template <typename T, typename V>
__global__ void __launch_bounds__(128) schwarz_apply_kernel(SchwarzArgs s, BgsArgs a) {
    __shared__ T sr[4][kSdMaxM];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = s.agg_lo + blockIdx.x * 4 + warp;
    const bool act = I < s.agg_hi;  // uniform per warp
    const int fb = s.fb, B = s.b;
    pdl_wait();
    pdl_trigger();
    if (!act) return;
    const int s0 = __ldg(s.sd_ptr + I), cnt = __ldg(s.sd_ptr + I + 1) - s0, m = cnt * fb;
    const T* __restrict__ rf = static_cast<const T*>(s.rf);
    for (int e = lane; e < m; e += 32) {
        const int p = e / fb, c = e - p * fb;
        sr[warp][e] = rf[(size_t)__ldg(s.sd_nodes + s0 + p) * fb + c];
    }
    __syncwarp();
    const int q = I * s.nfs + (s.nfs > 1 ? a.field : 0);
    const int m0 = __ldg(s.agg_ptr + I);
    const int own = (__ldg(s.agg_ptr + I + 1) - m0) * fb;
    const V* __restrict__ Xq = static_cast<const V*>(s.X) + __ldg(s.x_off + q);
    const T* __restrict__ x_in = static_cast<const T*>(a.x_in);
    const T* __restrict__ uc = static_cast<const T*>(a.uc);
    T* __restrict__ x_out = static_cast<T*>(a.x_out);
    for (int t = lane; t < own; t += 32) {
        T acc = T(0);
#pragma unroll 4
        for (int c = 0; c < m; ++c) acc = fma((T)Xq[(size_t)c * own + t], sr[warp][c], acc);
        const int i = __ldg(s.members + m0 + t / fb), cc = t % fb;
        const T om = a.omega_node ? static_cast<const T*>(a.omega_node)[(size_t)i * a.F + a.field] : T(a.omega);
        const int ag = (x_in && uc) ? __ldg(a.agg + i) : 0;
        for (int g = 0; g < a.F; ++g) {
            const size_t e = (size_t)i * B + g * fb + cc;
            T v = x_in ? x_in[e] : T(0);
            if (x_in && uc) v += uc[(size_t)ag * B + g * fb + cc];
            if (g == a.field) v = fma(om, acc, v);
            x_out[e] = v;
        }
    }
}

template <typename T>
int launch_field_residual(int b, int fb, int fm, int n, int field, const int* rp, const int* ci, const T* vals,
                          const T* x_in, const T* uc, const int* agg, const T* rhs, T* rf, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    const int grid = ceil_div((long)n * fb, 256);
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                         \
    case BB * 16 + FF: {                                                                                     \
        constexpr bool kFm = HasFm<T, BB, FF>::value;                                                       \
        const cudaError_t e =                                                                                \
            (fm && kFm) ? launch_k(field_residual_kernel<T, BB, FF, kFm>, grid, 256, 0, s, n, field, rp, ci, vals, \
                                   x_in, uc, agg, rhs, rf)                                                   \
                        : launch_k(field_residual_kernel<T, BB, FF, false>, grid, 256, 0, s, n, field, rp, ci,     \
                                   vals, x_in, uc, agg, rhs, rf);                                            \
        if (e != cudaSuccess) return BAMG_ECUDA;                                                             \
        break;                                                                                               \
    }
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}
template int launch_field_residual<double>(int, int, int, int, int, const int*, const int*, const double*,
                                           const double*, const double*, const int*, const double*, double*,
                                           cudaStream_t);
template int launch_field_residual<float>(int, int, int, int, int, const int*, const int*, const float*, const float*,
                                          const float*, const int*, const float*, float*, cudaStream_t);

template <typename T>
int launch_schwarz_apply(const SchwarzArgs& sa, const BgsArgs& a, cudaStream_t s) {
    const int nagg = sa.agg_hi - sa.agg_lo;
    if (nagg <= 0) return BAMG_OK;
    const int grid = ceil_div(nagg, 4);
    if (launch_k(schwarz_apply_kernel<T, T>, grid, 128, 0, s, sa, a) != cudaSuccess) return BAMG_ECUDA;
    return launched(1);
}
template int launch_schwarz_apply<double>(const SchwarzArgs&, const BgsArgs&, cudaStream_t);
template int launch_schwarz_apply<float>(const SchwarzArgs&, const BgsArgs&, cudaStream_t);

}  // namespace bamg
