// Device-side building blocks of the block Gauss-Seidel smoother of
// Algorithm 1 (Sec. 4.3.2) shared by the per-colour kernels (k_solve.cu) and
// the persistent sweep kernel (k_sweep.cu): vector loads with an optional
// L2-coherent path and the per-block accumulation of one field step.
#pragma once

#include "common.cuh"

namespace bamg {

// ---------------------------------------------------------------------------
// loads of B consecutive values of a vector (coherent variant for the tail)
// ---------------------------------------------------------------------------
template <typename T, int B, bool CG>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, T (&out)[B]) {
    if constexpr (!CG) {
        load_row<T, B>(p, out);
    } else {
        constexpr int bytes_row = B * (int)sizeof(T);
        if constexpr (sizeof(T) == 4 && bytes_row % 16 == 0) {
#pragma unroll
            for (int c = 0; c < B; c += 4) {
                float4 v = __ldcg(reinterpret_cast<const float4*>(p + c));
                out[c] = v.x;
                out[c + 1] = v.y;
                out[c + 2] = v.z;
                out[c + 3] = v.w;
            }
        } else if constexpr (bytes_row % 16 == 0 || (sizeof(T) == 4 && bytes_row % 8 == 0)) {
            using V2 = typename VecOf<T>::v2;
#pragma unroll
            for (int c = 0; c < B; c += 2) {
                V2 v = __ldcg(reinterpret_cast<const V2*>(p + c));
                out[c] = v.x;
                out[c + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int c = 0; c < B; ++c) out[c] = __ldcg(p + c);
        }
    }
}

template <typename T, bool CG>
__device__ __forceinline__ T ld1(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// one block of a field step of the smoother: acc += A_{f,*}[i,j] x_in,j (x_in
// plus P uc when fused), and acc += A_ff[i,j] x~_j when j precedes i in the
// colour order (x~ of later colours is stale and masked); arow = row f0 + r of
// the block.  Forced inline so that arow stays in registers.
// (CG: x~ read through L2 (it is written in the same launch); CGX: the same
// for x_in and uc, which only the tail kernel writes in the same launch)
template <typename T, int B, int FB, bool CG, bool CGX = CG>
__device__ __forceinline__ void bgs_block(const BgsArgs& a, const T* xt, const T* x_in, const T* uc, int j,
                                          const T (&arow)[B], bool lower, int ag, T& acc) {
    T tv[FB];
    if (lower) load_vec<T, FB, CG>(xt + (size_t)j * FB, tv);
    if (x_in) {
        T xv[B];
        load_vec<T, B, CGX>(x_in + (size_t)j * B, xv);
        if (uc) {
            T pv[B];
            load_vec<T, B, CGX>(uc + (size_t)ag * B, pv);
#pragma unroll
            for (int c = 0; c < B; ++c) xv[c] += pv[c];
        }
#pragma unroll
        for (int c = 0; c < B; ++c) acc = fma(arow[c], xv[c], acc);
    }
    if (lower) {
        // the field-f columns of the row, picked by selects over compile-time
        // register indices (an index computed from the field would put arow
        // in local memory)
#pragma unroll
        for (int c = 0; c < FB; ++c) {
            T av = arow[c];
#pragma unroll
            for (int ff = 1; ff < B / FB; ++ff) av = (ff == a.field) ? arow[ff * FB + c] : av;
            acc = fma(av, tv[c], acc);
        }
    }
}

// the blocks kf, kf + S, kf + 2S, ... (< k1) of one matrix row, accumulated
// in that order into acc (bgs_block per block).  Software-pipelined: the
// next block's colour flag, column and matrix row are loaded before the
// current block's gathers, so each step waits for one gather latency rather
// than the column load followed by its gather.  The first block (column jf,
// flag lowf, aggregate agf, row arf) is loaded by the caller, before its wait
// on the previous kernel; vb is the row's first block, VS the stride between
// blocks.  XIN: x_in is set (every block contributes; without it only blocks
// of lower colour do, and the others' rows are not loaded) -- a template
// flag, so that the loads of the next block do not wait on its colour flag.
template <typename T, int B, int FB, bool CG, int S, bool XIN>
__device__ __forceinline__ void bgs_walk_x(const BgsArgs& a, const T* xt, const T* x_in, const T* uc,
                                           const T* __restrict__ vb, int VS, int k0, int kf, int k1, int jf,
                                           bool lowf, int agf, const T (&arf)[B], T& acc) {
    int j = jf, ag = agf;
    bool lw = lowf;
    T ar[B];
#pragma unroll
    for (int c = 0; c < B; ++c) ar[c] = arf[c];
#pragma unroll 2
    for (int k = kf;; k += S) {
        const int kn = k + S;
        const bool more = kn < k1;
        bool lwn = false;
        int jn = 0;
        T an[B];
        if (more) {
            lwn = __ldg(a.lowk + kn) != 0;
            jn = __ldg(a.ci + kn);
            if (XIN || lwn) load_row<T, B>(vb + (size_t)(kn - k0) * VS, an);
        }
        if (XIN || lw) bgs_block<T, B, FB, CG>(a, xt, XIN ? x_in : nullptr, XIN ? uc : nullptr, j, ar, lw, ag, acc);
        if (!more) break;
        j = jn;
        lw = lwn;
        if (XIN && uc) ag = __ldg(a.agg + jn);
#pragma unroll
        for (int c = 0; c < B; ++c) ar[c] = an[c];
    }
}

template <typename T, int B, int FB, bool CG, int S>
__device__ __forceinline__ void bgs_walk(const BgsArgs& a, const T* xt, const T* x_in, const T* uc,
                                         const T* __restrict__ vb, int VS, int k0, int kf, int k1, int jf,
                                         bool lowf, int agf, const T (&arf)[B], T& acc) {
    if (x_in)
        bgs_walk_x<T, B, FB, CG, S, true>(a, xt, x_in, uc, vb, VS, k0, kf, k1, jf, lowf, agf, arf, acc);
    else
        bgs_walk_x<T, B, FB, CG, S, false>(a, xt, x_in, uc, vb, VS, k0, kf, k1, jf, lowf, agf, arf, acc);
}

}  // namespace bamg
