// One colour of one field step of the block Gauss-Seidel smoother
// (Algorithm 1, Sec. 4.3.2) with the matrix rows staged in shared memory by
// asynchronous copies, for levels far larger than L2.
//
// The thread-per-row kernels read every block row straight from HBM, and
// each thread's chain of column index -> gather -> row leaves few bytes in
// flight: on the 3D 64^3 level 0 a colour launch keeps HBM 41% busy while
// most warps wait on long-scoreboard stalls.  Here every CTA owns a run of
// the colour's nodes, cut into batches of kNodes nodes.  The FB * G threads
// of a node copy its values (the field's part in the field-major layout),
// column indices and lower-colour flags into the node's shared-memory slot
// with 16-byte cp.async copies (no registers held while they fly; one commit
// group per batch), kStages batches ahead of the batch the CTA computes from
// shared memory.  The copies of the first batches are issued before the wait
// on the previous kernel (the matrix is fixed during a cycle), so they overlap
// its tail.  (A first version with one bulk copy per node and region spent
// most of its time in the copy engine's per-request cost: three requests of
// 32 B to 1.7 KB per node.)  Measured on GB300: about as fast as the warp
// kernel on L2-resident levels, and slower than the four-lanes kernel on the
// 3D 64^3 level 0 (40 against 21 us per colour): the compute phase, whose
// gathers of the iterate wait on L2, bounds a batch at the occupancy that the
// slots leave (two CTAs per SM).  The autotuner keeps whichever is faster.
//
// Copies move whole 16-byte units from 16-byte-aligned addresses: each range
// is widened to [floor16(start), ceil16(end)) and read from its offset inside
// the slot (the library pads every buffer by 64 bytes, so the widened range
// stays inside its allocation).  Slot offsets are multiples of 16, so a value
// keeps its address modulo 16 and the vector loads of load_row stay aligned.
// The CTA waits for all its copies before it leaves.
//
// Lanes, order of the sums and the update are those of the four-lanes-per-row
// kernel (bgs_tpr_kernel with G = 4), so both give the same values bit for bit.
#include "bgs_body.cuh"
#include "common.cuh"

namespace bamg {

constexpr int kStagedStages = 3;

template <int FB>
struct StagedShape {
    static constexpr int kThreads = RowThreads<FB>::kThreads;
    static constexpr int kG = 4;                             // lanes per scalar row
    static constexpr int kNodes = kThreads / (FB * kG);      // nodes per batch
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// byte layout of one node's slot: values, then columns, then flags, each
// region rounded up to 16 bytes with 16 bytes of slack for the widening
struct StagedSlot {
    int vals, cols, flags, total;
};
__host__ __device__ inline StagedSlot staged_slot(int max_row, int row_bytes_per_block) {
    StagedSlot t;
    t.vals = ((max_row * row_bytes_per_block + 15) & ~15) + 16;
    t.cols = ((max_row * 4 + 15) & ~15) + 16;
    t.flags = ((max_row + 15) & ~15) + 16;
    t.total = t.vals + t.cols + t.flags;
    return t;
}

template <typename T, int B, int FB, bool FM>
__host__ __device__ constexpr int staged_block_bytes() {
    return (FM && HasFm<T, B, FB>::value) ? FB * B * (int)sizeof(T) : B * B * (int)sizeof(T);
}

// 16-byte asynchronous copy global -> shared (both 16-byte aligned), and
// its commit / wait
__device__ __forceinline__ void cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// the FB * G threads of node slot nloc copy the node's three widened ranges
// in 16-byte pieces (w = the thread's index among them)
template <typename T, int B, int FB, bool FM, int NTN>
__device__ __forceinline__ void stage_node(const BgsArgs& a, int i, char* slot, const StagedSlot& ts, int w,
                                           int* err) {
    const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1), len = k1 - k0;
    constexpr int RB = staged_block_bytes<T, B, FB, FM>();
    const size_t va = (FM && HasFm<T, B, FB>::value)
                          ? ((size_t)k0 * B * B + (size_t)a.field * len * FB * B) * sizeof(T)
                          : (size_t)k0 * B * B * sizeof(T);
    const size_t vb = va + (size_t)len * RB;
    const size_t va16 = va & ~(size_t)15, vb16 = (vb + 15) & ~(size_t)15;
    const size_t ca16 = ((size_t)k0 * 4) & ~(size_t)15, cb16 = ((size_t)k1 * 4 + 15) & ~(size_t)15;
    const size_t la16 = (size_t)k0 & ~(size_t)15, lb16 = ((size_t)k1 + 15) & ~(size_t)15;
    const char* vs = static_cast<const char*>(a.vals) + va16;
    const char* cs = reinterpret_cast<const char*>(a.ci) + ca16;
    const char* ls = reinterpret_cast<const char*>(a.lowk) + la16;
    const int nv = (int)((vb16 - va16) >> 4), nc = (int)((cb16 - ca16) >> 4), nl = (int)((lb16 - la16) >> 4);
    // every copy starts on 16 bytes at both ends and stays in its region of
    // the slot (by construction; checked, and skipped with an error if not)
    if (((reinterpret_cast<uintptr_t>(vs) | reinterpret_cast<uintptr_t>(cs) | reinterpret_cast<uintptr_t>(ls)) & 15) ||
        (smem_u32(slot) & 15) || nv * 16 > ts.vals || nc * 16 > ts.cols || nl * 16 > ts.flags) {
        set_error(err, kDevBadPattern);
        return;
    }
    for (int c = w; c < nv; c += NTN) cp16(slot + c * 16, vs + (size_t)c * 16);
    for (int c = w; c < nc; c += NTN) cp16(slot + ts.vals + c * 16, cs + (size_t)c * 16);
    for (int c = w; c < nl; c += NTN) cp16(slot + ts.vals + ts.cols + c * 16, ls + (size_t)c * 16);
}

template <typename T, int B, int FB, bool FM>
__global__ void __launch_bounds__(StagedShape<FB>::kThreads) bgs_staged_kernel(BgsArgs a, int max_row, int batches_per_cta,
                                                                         int* err) {
    constexpr int G = StagedShape<FB>::kG, NB = StagedShape<FB>::kNodes;
    constexpr int RB = staged_block_bytes<T, B, FB, FM>();
    extern __shared__ __align__(128) char smem_raw[];
    // the slots start on a 128-byte boundary of the shared window (the launch
    // adds 128 bytes for this)
    char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ T sh_t[NB * FB];
    const StagedSlot ts = staged_slot(max_row, RB);
    const int tid = threadIdx.x;
    const int nloc = tid / (FB * G);
    const int w = tid - nloc * (FB * G);
    const int r = w / G, sl = w - r * G;
    const int f0 = a.field * FB;
    const T* __restrict__ x_in = static_cast<const T*>(a.x_in);
    const T* __restrict__ uc = static_cast<const T*>(a.uc);
    const T* __restrict__ xt = static_cast<const T*>(a.xt);
    const long first = (long)blockIdx.x * batches_per_cta * NB;
    long nbatch = ((long)a.n_in_colour - first + NB - 1) / NB;
    if (nbatch > batches_per_cta) nbatch = batches_per_cta;
    if (nbatch < 0) nbatch = 0;
    // batch t into stage t % kStagedStages: node slot nloc by its FB * G threads;
    // one commit group per batch (empty past the last), so that group t is
    // complete once all but the kStagedStages - 1 latest groups are
    auto issue = [&](long t) {
        if (t < nbatch) {
            const long q = first + t * NB + nloc;
            if (q < a.n_in_colour)
                stage_node<T, B, FB, FM, FB * G>(a, __ldg(a.nodes + q),
                                                 smem + ((size_t)(t % kStagedStages) * NB + nloc) * ts.total, ts, w,
                                                 err);
        }
        cp_commit();
    };
    for (long t = 0; t < kStagedStages; ++t) issue(t);  // the matrix is fixed: before the wait
    pdl_wait();
    pdl_trigger();
    for (long t = 0; t < nbatch; ++t) {
        const int st = (int)(t % kStagedStages);
        cp_wait<kStagedStages - 1>();  // this thread's pieces of batch t have landed
        __syncthreads();            // and everyone's
        const long q = first + t * NB + nloc;
        const bool act = q < a.n_in_colour;
        int i = 0;
        T acc = T(0);
        if (act) {
            i = __ldg(a.nodes + q);
            const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1), len = k1 - k0;
            const char* slot = smem + ((size_t)st * NB + nloc) * ts.total;
            const size_t va = (FM && HasFm<T, B, FB>::value)
                                  ? ((size_t)k0 * B * B + (size_t)a.field * len * FB * B) * sizeof(T)
                                  : (size_t)k0 * B * B * sizeof(T);
            const T* vrow0 = reinterpret_cast<const T*>(slot + (va & 15));
            const int* crow = reinterpret_cast<const int*>(slot + ts.vals + (((size_t)k0 * 4) & 15));
            const unsigned char* lrow =
                reinterpret_cast<const unsigned char*>(slot + ts.vals + ts.cols + ((size_t)k0 & 15));
            // this lane's row of block kk: block-major rows f0 + r of B*B
            // blocks, or rows r of the field's FB*B blocks (field-major)
            constexpr int VS = RB / (int)sizeof(T);
            const int roff = (FM && HasFm<T, B, FB>::value) ? r * B : (f0 + r) * B;
#pragma unroll 2
            for (int kk = sl; kk < len; kk += G) {
                const bool lower = lrow[kk] != 0;
                if (!x_in && !lower) continue;
                const int j = crow[kk];
                T arow[B];
                load_row<T, B>(vrow0 + (size_t)kk * VS + roff, arow);
                bgs_block<T, B, FB, false>(a, xt, x_in, uc, j, arow, lower, (x_in && uc) ? __ldg(a.agg + j) : 0,
                                           acc);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (sl == 0) sh_t[nloc * FB + r] = act ? static_cast<const T*>(a.rhs)[(size_t)i * B + f0 + r] - acc : T(0);
        __syncthreads();  // the row sums are in sh_t; every thread is done with stage st
        if (act && sl == 0) {
            const T* D = static_cast<const T*>(a.dinv) + ((size_t)i * a.F + a.field) * FB * FB + (size_t)r * FB;
            T xn = T(0);
#pragma unroll
            for (int c = 0; c < FB; ++c) xn = fma(__ldg(D + c), sh_t[nloc * FB + c], xn);
            static_cast<T*>(a.xt)[(size_t)i * FB + r] = xn;
            T* __restrict__ x_out = static_cast<T*>(a.x_out);
            const T om =
                a.omega_node ? static_cast<const T*>(a.omega_node)[(size_t)i * a.F + a.field] : T(a.omega);
            const int ag = (x_in && uc) ? __ldg(a.agg + i) : 0;
            for (int m = 0; m < a.F; ++m) {
                const size_t e = (size_t)i * B + m * FB + r;
                T v = x_in ? x_in[e] : T(0);
                if (x_in && uc) v += uc[(size_t)ag * B + m * FB + r];
                if (m == a.field) v = fma(om, xn, v);
                x_out[e] = v;
            }
        }
        issue(t + kStagedStages);  // refill stage st (its reads ended at the barrier above)
        __syncthreads();        // sh_t is reused by the next batch
    }
    cp_wait<0>();  // nothing in flight when the CTA leaves
}

template <typename T, int B, int FB, bool FM>
static int launch_staged_instance(const BgsArgs& a, int max_row, int* err, cudaStream_t s) {
    constexpr int NT = StagedShape<FB>::kThreads, NB = StagedShape<FB>::kNodes;
    const StagedSlot ts = staged_slot(max_row, staged_block_bytes<T, B, FB, FM>());
    const size_t smem = (size_t)kStagedStages * NB * ts.total + 128;
    if (smem > 200 * 1024) return BAMG_EUNSUPPORTED;
    static int attr_set = 0;  // the largest dynamic size requested so far
    if ((int)smem > attr_set) {
        if (cudaFuncSetAttribute(bgs_staged_kernel<T, B, FB, FM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024) != cudaSuccess)
            return BAMG_ECUDA;
        attr_set = 200 * 1024;
    }
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                     cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bgs_staged_kernel<T, B, FB, FM>, NT, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return BAMG_EUNSUPPORTED;
    // one wave of resident CTAs, each a contiguous run of batches
    const long batches = (a.n_in_colour + NB - 1) / NB;
    const long ctas_max = (long)sms * per_sm;
    const int per_cta = (int)((batches + ctas_max - 1) / ctas_max);
    const int grid = (int)((batches + per_cta - 1) / per_cta);
    if (launch_k(bgs_staged_kernel<T, B, FB, FM>, grid, NT, smem, s, a, max_row, per_cta, err) != cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}

template <typename T>
int launch_bgs_colour_staged(int b, int fb, const BgsArgs& a, int max_row, int* err, cudaStream_t s) {
    if (a.n_in_colour <= 0) return BAMG_OK;
    // whole blocks are staged: one field of several only in the field-major layout
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                     \
    case BB * 16 + FF: {                                                                                 \
        constexpr bool kFm = HasFm<T, BB, FF>::value;                                                   \
        if (BB != FF && !(a.fm && kFm)) return BAMG_EUNSUPPORTED;                                        \
        return (a.fm && kFm) ? launch_staged_instance<T, BB, FF, kFm>(a, max_row, err, s)                   \
                             : launch_staged_instance<T, BB, FF, false>(a, max_row, err, s);                \
    }
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
}
template int launch_bgs_colour_staged<double>(int, int, const BgsArgs&, int, int*, cudaStream_t);
template int launch_bgs_colour_staged<float>(int, int, const BgsArgs&, int, int*, cudaStream_t);

// the largest number of stored blocks in a row
__global__ void row_len_max_kernel(int n, const int* __restrict__ rp, int* __restrict__ out) {
    int m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, rp[i + 1] - rp[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}
int launch_row_len_max(int n, const int* rp, int* out, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    BAMG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int), s));
    row_len_max_kernel<<<ceil_div(n, 256) < 1024 ? ceil_div(n, 256) : 1024, 256, 0, s>>>(n, rp, out);
    return launched(1);
}

}  // namespace bamg
