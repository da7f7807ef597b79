// Dense FP32 factorisation and inverse of the coarsest-level matrix on the
// 5th-generation tensor cores (the coarsest direct solve of the V-cycle,
// Sec. 4.1, for FP32 cycles).
//
//   LU:       blocked right-looking LU with partial pivoting, panels of 16
//             columns.  Per panel: one CTA factors the panel with its rows in
//             registers (pivot = largest |value|, ties to the lowest row), the
//             panel's row swaps are applied to the other columns and
//             U12 = L11^-1 A12 is formed (one thread per column), and the
//             trailing matrix takes A22 -= L21 U12 as a tcgen05 GEMM.
//   inverse:  A^-1 = U^-1 L^-1 P by blocked triangular solves on the identity
//             (blocks of 128 rows): the diagonal blocks' inverses first, then
//             per block one GEMM that applies a diagonal inverse and one that
//             updates the remaining blocks, all on the tensor cores.
//
// Tensor-core arithmetic: tcgen05.mma kind::tf32 reads 19-bit operands, so
// each FP32 operand x is split into hi = tf32(x) and lo = tf32(x - hi) and a
// product is accumulated as hi*hi + hi*lo + lo*hi in the FP32 accumulator
// (the "3xTF32" error-compensated split of Ootomo and Yokota, 2022), an error
// of a few units of FP32 rounding per product.
//
// GEMM kernel layout: one CTA per 128 x 128 output tile, 256 threads.  All
// threads stage K-slices of 32 of the A tile (128 x 32) and of the B tile
// (stored N x K) into shared memory in the canonical K-major, non-swizzled
// layout of the tensor core (8-row x 16-byte core matrices), split into hi and
// lo; one elected thread issues the MMAs into a 128 x 128 FP32 accumulator in
// tensor memory (128 columns) and commits them to an mbarrier; two stages
// alternate so that the staging of slice s+1 overlaps the MMAs of slice s
// (a product with K <= 32 has one slice, one stage, and three CTAs per SM).
// The epilogue reads the accumulator with tcgen05.ld (warp w reads lanes
// 32 (w mod 4) ..) and writes C = D + sign * A B.  Every wait on an mbarrier
// is bounded: on time-out the kernel records kDevTimeout, waits (bounded) for
// its last commit, frees its tensor memory and returns.
#include "common.cuh"

namespace bamg {

namespace {

constexpr int kTcTile = 128;      // M = N of one MMA tile
constexpr int kTcK = 32;          // K per staged slice
constexpr int kTcThreads = 256;   // staging threads (and epilogue)
constexpr int kTcOperand = kTcTile * kTcK * 4;       // bytes of one split operand tile (16 KB)
constexpr int kTcStage = 4 * kTcOperand;             // A hi, A lo, B hi, B lo
constexpr int kTcSmem = 2 * kTcStage + 1024;         // two stages + alignment slack
constexpr long kTcSpins = 1L << 22;                  // bounded mbarrier waits
constexpr int kPanel = 16;        // LU panel width
constexpr int kPanelThreads = 512;
constexpr int kPanelRPT = 4;                         // rows per thread
constexpr int kPanelRows = kPanelRPT * kPanelThreads;  // rows a panel CTA holds (2048)
constexpr int kInvBlock = 128;    // block of the inverse's triangular solves

#define TRY_OK(expr)                    \
    do {                                \
        const int st_ = (expr);         \
        if (st_ != BAMG_OK) return st_; \
    } while (0)

// ---------------------------------------------------------------------------
// PTX wrappers (tcgen05, mbarrier, proxy fences)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the completion of the phase of the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (long i = 0; i < kTcSpins; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// whole warp: allocate ncols columns of tensor memory, address to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D[tmem] (+)= A[smem] * B[smem], kind::tf32, one CTA
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread is done
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// round to the nearest TF32 value (low 13 mantissa bits cleared)
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance of
// core matrices adjacent in K, sbo = of core matrices adjacent in M/N
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this tensor-core generation
    return d;                // base offset 0, relative lbo, no swizzle
}
// instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// byte offset of element (row, kk) of a 128 x 32 K-major tile: core matrices
// of 8 rows x 4 elements (128 bytes), adjacent in K 128 bytes apart (lbo),
// adjacent in rows 1024 bytes apart (sbo)
__device__ __forceinline__ uint32_t tile_off(int row, int kk) {
    return (uint32_t)((row >> 3) * 1024 + (kk >> 2) * 128 + (row & 7) * 16 + (kk & 3) * 4);
}
constexpr uint32_t kLbo = 128, kSbo = 1024;

}  // namespace

// C[m x n] = D + sign * A[m x k] B[k x n] (row-major FP32; D may be C, or
// null for zero).  Grid (ceil(n/128), ceil(m/128)).
struct TcGemmArgs {
    int m, n, k;
    const float* A;
    int lda;
    const float* B;
    int ldb;
    const float* D;
    int ldd;
    float* C;
    int ldc;
    float sign;
    int* err;
};

__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(TcGemmArgs g) {
    extern __shared__ __align__(1024) unsigned char tc_sh[];
    __shared__ uint64_t bar[2];
    __shared__ uint32_t s_taddr;
    // operand tiles on a 1024-byte boundary
    unsigned char* base = tc_sh + ((1024u - (smem_u32(tc_sh) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * kTcTile, n0 = blockIdx.x * kTcTile;
    if (warp == 0) tmem_alloc(&s_taddr, kTcTile);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    pdl_wait();
    constexpr uint32_t kIdesc = idesc_tf32(kTcTile, kTcTile);
    const int nk = (g.k + kTcK - 1) / kTcK;
    int committed = 0;
    bool fail = false;
    for (int kt = 0; kt < nk; ++kt) {
        const int st = nk > 1 ? (kt & 1) : 0;  // one K slice: one stage (a smaller launch)
        unsigned char* sa_hi = base + st * kTcStage;
        unsigned char* sa_lo = sa_hi + kTcOperand;
        unsigned char* sb_hi = sa_hi + 2 * kTcOperand;
        unsigned char* sb_lo = sa_hi + 3 * kTcOperand;
        const int kb = kt * kTcK;
        // this slice's operands into registers first (every load in flight
        // at once, and before the wait for the stage's previous MMAs)
        // A: rows (tid / 8) + 32 i, K chunk (tid mod 8) of 4 elements;
        // B, stored N x K: column tid mod 128, K chunks (tid / 128) + 2 i
        float ea[4][4], eb[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gr = m0 + (tid >> 3) + 32 * i, kc = (tid & 7) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int gk = kb + kc + q;
                ea[i][q] = (gr < g.m && gk < g.k) ? __ldcg(g.A + (size_t)gr * g.lda + gk) : 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gc = n0 + (tid & (kTcTile - 1)), kc = ((tid >> 7) + 2 * i) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int gk = kb + kc + q;
                eb[i][q] = (gc < g.n && gk < g.k) ? __ldcg(g.B + (size_t)gk * g.ldb + gc) : 0.f;
            }
        }
        // the MMAs that read this stage two slices ago are done
        if (kt >= 2 && !mbar_wait(&bar[st], ((kt - 2) >> 1) & 1)) fail = true;
        if (__syncthreads_or(fail)) {
            fail = true;
            break;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = (tid >> 3) + 32 * i, kc = (tid & 7) * 4;
            float4 hi, lo;
            hi.x = to_tf32(ea[i][0]); lo.x = to_tf32(ea[i][0] - hi.x);
            hi.y = to_tf32(ea[i][1]); lo.y = to_tf32(ea[i][1] - hi.y);
            hi.z = to_tf32(ea[i][2]); lo.z = to_tf32(ea[i][2] - hi.z);
            hi.w = to_tf32(ea[i][3]); lo.w = to_tf32(ea[i][3] - hi.w);
            *reinterpret_cast<float4*>(sa_hi + tile_off(row, kc)) = hi;
            *reinterpret_cast<float4*>(sa_lo + tile_off(row, kc)) = lo;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int col = tid & (kTcTile - 1), kc = ((tid >> 7) + 2 * i) * 4;
            float4 hi, lo;
            hi.x = to_tf32(eb[i][0]); lo.x = to_tf32(eb[i][0] - hi.x);
            hi.y = to_tf32(eb[i][1]); lo.y = to_tf32(eb[i][1] - hi.y);
            hi.z = to_tf32(eb[i][2]); lo.z = to_tf32(eb[i][2] - hi.z);
            hi.w = to_tf32(eb[i][3]); lo.w = to_tf32(eb[i][3] - hi.w);
            *reinterpret_cast<float4*>(sb_hi + tile_off(col, kc)) = hi;
            *reinterpret_cast<float4*>(sb_lo + tile_off(col, kc)) = lo;
        }
        fence_async_smem();  // the generic-proxy stores, visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < kTcK / 8; ++s) {  // K = 8 per MMA: two core matrices along K
                const uint32_t off = (uint32_t)s * 2u * kLbo;
                const uint64_t ah = smem_desc(smem_u32(sa_hi) + off, kLbo, kSbo);
                const uint64_t al = smem_desc(smem_u32(sa_lo) + off, kLbo, kSbo);
                const uint64_t bh = smem_desc(smem_u32(sb_hi) + off, kLbo, kSbo);
                const uint64_t bl = smem_desc(smem_u32(sb_lo) + off, kLbo, kSbo);
                tc_mma_tf32(taddr, al, bh, kIdesc, (kt > 0 || s > 0) ? 1u : 0u);  // small terms first
                tc_mma_tf32(taddr, ah, bl, kIdesc, 1u);
                tc_mma_tf32(taddr, ah, bh, kIdesc, 1u);
            }
            tc_commit(&bar[st]);
        }
        ++committed;
    }
    pdl_trigger();
    // every MMA done (the last commit covers all earlier ones)
    if (committed > 0 && !mbar_wait(&bar[(committed - 1) & 1], ((committed - 1) >> 1) & 1)) fail = true;
    fail = __syncthreads_or(fail);
    if (fail) {
        if (tid == 0) set_error(g.err, kDevTimeout);
    } else {
        tc_fence_after();
        // accumulator -> shared memory, then D and C by whole rows, coalesced
        // (the stage buffers are free: every MMA is done)
        // (rows of kTcTile floats, column c of row r at (c + r) mod kTcTile:
        // the lanes of a warp hit distinct banks both when they write one row
        // each and when they read one row together; 64 KB, one stage)
        float* tile = reinterpret_cast<float*>(base);
        constexpr int TS = kTcTile;
        const int lane_base = (warp & 3) * 32;  // accumulator lanes this warp may read
        const int col_base = (warp >> 2) * (kTcTile / 2);
        const int lr = lane_base + (tid & 31);
#pragma unroll 1
        for (int c0 = 0; c0 < kTcTile / 2; c0 += 32) {
            float v[32];
            if (committed > 0) {
                tmem_ld32(taddr + ((uint32_t)lane_base << 16) + (uint32_t)(col_base + c0), v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) tile[lr * TS + ((col_base + c0 + j + lr) & (kTcTile - 1))] = v[j];
        }
        __syncthreads();
        // D and C by whole rows (warp w: rows w, w + 8, ...), coalesced; every
        // D value is loaded before the first store (C may alias D)
        const int lane = tid & 31;
        constexpr int RPW = kTcTile / (kTcThreads / 32);  // rows per warp
        float dv[RPW][kTcTile / 32];
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const int row = m0 + warp + i * (kTcThreads / 32);
#pragma unroll
            for (int q = 0; q < kTcTile / 32; ++q) {
                const int gc = n0 + q * 32 + lane;
                dv[i][q] = (g.D && row < g.m && gc < g.n) ? g.D[(size_t)row * g.ldd + gc] : 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const int r = warp + i * (kTcThreads / 32), row = m0 + r;
#pragma unroll
            for (int q = 0; q < kTcTile / 32; ++q) {
                const int col = q * 32 + lane, gc = n0 + col;
                if (row < g.m && gc < g.n)
                    g.C[(size_t)row * g.ldc + gc] = fmaf(g.sign, tile[r * TS + ((col + r) & (kTcTile - 1))], dv[i][q]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_free(taddr, kTcTile);
}

namespace {
cudaError_t launch_pdl(const void* fn, dim3 grid, dim3 block, size_t smem, cudaStream_t s, void** args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}
}  // namespace

namespace {
int launch_tc_gemm_args(const TcGemmArgs& g, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        BAMG_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
        attr_set = true;
    }
    TcGemmArgs a = g;
    void* args[] = {&a};
    const dim3 grid((unsigned)((g.n + kTcTile - 1) / kTcTile), (unsigned)((g.m + kTcTile - 1) / kTcTile));
    // one K slice needs one stage: three CTAs per SM instead of one
    const size_t smem = g.k > kTcK ? (size_t)kTcSmem : (size_t)(kTcStage + 1024);
    if (launch_pdl((const void*)tc_gemm_kernel, grid, dim3(kTcThreads), smem, s, args) != cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}

}  // namespace

int launch_tc_gemm(int m, int n, int k, const float* A, int lda, const float* B, int ldb, const float* D, int ldd,
                   float* C, int ldc, float sign, int* err, cudaStream_t s) {
    if (m <= 0 || n <= 0) return BAMG_OK;
    TcGemmArgs g{};
    g.m = m;
    g.n = n;
    g.k = k;
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.D = D;
    g.ldd = ldd;
    g.C = C;
    g.ldc = ldc;
    g.sign = sign;
    g.err = err;
    return launch_tc_gemm_args(g, s);
}

// ---------------------------------------------------------------------------
// LU panel: columns p0 .. p0 + nb of rows p0 .. nd (nd - p0 <= 2048), one CTA of
// kPanelThreads threads, thread t holding rows t, t + kPanelThreads, ... of the
// panel in registers.  Each row's registers are a window that starts at the
// current column: per column j the largest |window[0]| among the rows not yet
// chosen (ties to the lower row) is the pivot; each warp publishes its best
// candidate's window in shared memory, so one barrier per column makes the
// pivot row known to all; every other row stores its multiplier l (its
// window[0] / pivot) and shifts its window by one while updating it
// (window[c] = window[c + 1] - l pivot[c + 1]), so the column loop runs with
// compile-time register indices and is not unrolled.  A row chosen as pivot
// stores its window (the U entries) and stops.  The finished rows collect in
// shared memory.  At the end the choices are replayed as the sequential row
// swaps of the panel (position p0 + j <-> the pivot's position), the rows are
// written back at their new positions, perm (original row at each position)
// follows the swaps, and mv records the row moves for the other columns:
// mv[j] (j < nb) = the row whose values go to position p0 + j, mv[kPanel] =
// the number of other positions that change, then (destination, source)
// pairs.
// ---------------------------------------------------------------------------
constexpr float kTcTiny = 1e-9f;  // pivot below kTcTiny * ||A||_inf: singular (as the CUDA-core FP32 LU)
constexpr int kStageLd = kPanel + 1;  // padded rows of the finished-row stage
// dynamic shared memory of the panel kernel for R rows
constexpr size_t panel_smem(int R) { return (size_t)R * (kStageLd * sizeof(float) + 3 * sizeof(int)); }

__global__ void __launch_bounds__(kPanelThreads, 1) tc_panel_kernel(int nd, int p0, float* __restrict__ a,
                                                                    int* __restrict__ mv, int* __restrict__ perm,
                                                                    const float* __restrict__ norm, int* err) {
    extern __shared__ __align__(16) float pan_sh[];  // stage[R][kStageLd], where_[R], at_[R], perm_s[R]
    constexpr int NW = kPanelThreads / 32;
    // per column (double-buffered by its parity): each warp's best candidate
    // key, its row and the row's window
    __shared__ float cand[2][NW][kPanel];
    __shared__ unsigned red_k[2][NW];
    __shared__ unsigned red_r[2][NW];
    __shared__ int pl[kPanel];
    __shared__ int n_mv;
    pdl_wait();
    const int R = nd - p0, nb = min(kPanel, R);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    float* stage = pan_sh;
    int* where_ = reinterpret_cast<int*>(pan_sh + (size_t)R * kStageLd);
    int* at_ = where_ + R;
    int* perm_s = at_ + R;
    float v[kPanelRPT][kPanel];
    bool done[kPanelRPT];
    const bool vec = (nd & 3) == 0 && nb == kPanel;  // rows of 16 floats on 16-byte boundaries
#pragma unroll
    for (int rr = 0; rr < kPanelRPT; ++rr) {
        const int r = t + rr * kPanelThreads;
        done[rr] = r >= R;
        const float* src = a + (size_t)(p0 + r) * nd + p0;
        if (vec && r < R) {
#pragma unroll
            for (int c = 0; c < kPanel; c += 4) {
                const float4 q = *reinterpret_cast<const float4*>(src + c);
                v[rr][c] = q.x;
                v[rr][c + 1] = q.y;
                v[rr][c + 2] = q.z;
                v[rr][c + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int c = 0; c < kPanel; ++c) v[rr][c] = (r < R && c < nb) ? src[c] : 0.f;
        }
    }
    const float nrm = norm[0];
#pragma unroll 1
    for (int j = 0; j < nb; ++j) {
        const int buf = j & 1;
        // candidate key: the bits of |value| + 1 (non-negative floats order
        // as unsigned integers; 0 = no candidate), ties to the lower row
        unsigned key = 0u, row = 0xFFFFFFFFu;
        int own = -1;
#pragma unroll
        for (int rr = 0; rr < kPanelRPT; ++rr) {
            const unsigned k = __float_as_uint(fabsf(v[rr][0])) + 1u;
            if (!done[rr] && k > key) {
                key = k;
                row = (unsigned)(t + rr * kPanelThreads);
                own = rr;
            }
        }
        unsigned m = __reduce_max_sync(0xffffffffu, key);
        unsigned rmin = __reduce_min_sync(0xffffffffu, key == m ? row : 0xFFFFFFFFu);
        if (lane == 0) {
            red_k[buf][w] = m;
            red_r[buf][w] = rmin;
        }
        if (m != 0u && rmin == row) {  // this lane holds the warp's candidate: publish its window
#pragma unroll
            for (int c = 0; c < kPanel; ++c) {
                float x = v[0][c];
#pragma unroll
                for (int rr = 1; rr < kPanelRPT; ++rr) x = own == rr ? v[rr][c] : x;
                cand[buf][w][c] = x;
            }
        }
        __syncthreads();
        key = lane < NW ? red_k[buf][lane] : 0u;
        row = lane < NW ? red_r[buf][lane] : 0xFFFFFFFFu;
        m = __reduce_max_sync(0xffffffffu, key);
        rmin = __reduce_min_sync(0xffffffffu, key == m ? row : 0xFFFFFFFFu);
        const int wi = __ffs(__ballot_sync(0xffffffffu, key == m && row == rmin)) - 1;
        const int bi = (int)rmin;
        if (t == 0) {
            pl[j] = bi;
            const float best = m == 0u ? -1.f : __uint_as_float(m - 1u);
            if (!(best >= kTcTiny * nrm) || nrm == 0.f || bi >= R) set_error(err, kDevSingularCoarse);
        }
        const float* prow = cand[buf][wi];
        const float rp = __frcp_rn(prow[0]);
        float pv[kPanel - 1];
#pragma unroll
        for (int c = 0; c < kPanel - 1; ++c) pv[c] = prow[c + 1];
#pragma unroll
        for (int rr = 0; rr < kPanelRPT; ++rr) {
            const int r = t + rr * kPanelThreads;
            if (done[rr]) continue;
            float* srow = stage + (size_t)r * kStageLd + j;
            if (r == bi) {  // the pivot row: its window is row j of U
                done[rr] = true;
#pragma unroll
                for (int c = 0; c < kPanel; ++c)
                    if (c < kPanel - j) srow[c] = v[rr][c];
            } else {
                const float l = v[rr][0] * rp;
                srow[0] = l;
#pragma unroll
                for (int c = 0; c < kPanel - 1; ++c) v[rr][c] = fmaf(-l, pv[c], v[rr][c + 1]);
                v[rr][kPanel - 1] = 0.f;
            }
        }
    }
    __syncthreads();
    for (int r = t; r < R; r += kPanelThreads) {
        where_[r] = r;
        at_[r] = r;
        perm_s[r] = perm[p0 + r];
    }
    __syncthreads();
    if (t == 0)
        for (int j = 0; j < nb; ++j) {
            const int r = min(max(pl[j], 0), R - 1), q = where_[r], rj = at_[j];
            at_[j] = r;
            at_[q] = rj;
            where_[r] = j;
            where_[rj] = q;
            const int ps = perm_s[j];
            perm_s[j] = perm_s[q];
            perm_s[q] = ps;
        }
    if (t == 0) n_mv = 0;
    __syncthreads();
    // the moves for the other columns: the top positions, and the (at most
    // nb) positions below them that received a displaced row
    if (t < nb) mv[t] = p0 + at_[t];
    for (int x = nb + t; x < R; x += kPanelThreads)
        if (at_[x] != x) {
            const int k = atomicAdd(&n_mv, 1);
            if (k < kPanel) {
                mv[kPanel + 1 + 2 * k] = p0 + x;
                mv[kPanel + 2 + 2 * k] = p0 + at_[x];
            }
        }
    // finished rows to their new positions
    for (int r = t; r < R; r += kPanelThreads) {
        const float* srow = stage + (size_t)r * kStageLd;
        float* dst = a + (size_t)(p0 + where_[r]) * nd + p0;
        if (vec) {
#pragma unroll
            for (int c = 0; c < kPanel; c += 4)
                *reinterpret_cast<float4*>(dst + c) = make_float4(srow[c], srow[c + 1], srow[c + 2], srow[c + 3]);
        } else {
            for (int c = 0; c < nb; ++c) dst[c] = srow[c];
        }
    }
    for (int r = t; r < R; r += kPanelThreads) perm[p0 + r] = perm_s[r];
    __syncthreads();
    if (t == 0) mv[kPanel] = min(n_mv, kPanel);
    pdl_trigger();
}

// the panel's row moves on every column outside it (one thread per column:
// every source value is loaded before any store), then U12 = L11^-1 A12 on
// the panel's rows for the columns right of the panel (L11: unit lower, the
// panel's top nb x nb block)
__global__ void __launch_bounds__(256) tc_swap_trsm_kernel(int nd, int p0, float* __restrict__ a,
                                                           const int* __restrict__ mv) {
    __shared__ float l11[kPanel][kPanel + 1];
    __shared__ int s_mv[3 * kPanel + 1];
    pdl_wait();
    const int nb = min(kPanel, nd - p0), c0 = p0 + nb;
    const int t = threadIdx.x;
    for (int e = t; e < kPanel * kPanel; e += blockDim.x) {
        const int r = e / kPanel, c = e - r * kPanel;
        l11[r][c] = (r < nb && c < nb) ? a[(size_t)(p0 + r) * nd + p0 + c] : 0.f;
    }
    if (t < 3 * kPanel + 1) s_mv[t] = mv[t];
    __syncthreads();
    pdl_trigger();
    const int q = blockIdx.x * blockDim.x + t;
    if (q >= nd - nb) return;
    const int c = q < p0 ? q : q + nb;
    const int nm = s_mv[kPanel];
    float x[kPanel], y[kPanel];
#pragma unroll
    for (int j = 0; j < kPanel; ++j) x[j] = j < nb ? a[(size_t)s_mv[j] * nd + c] : 0.f;
#pragma unroll
    for (int k = 0; k < kPanel; ++k) y[k] = k < nm ? a[(size_t)s_mv[kPanel + 2 + 2 * k] * nd + c] : 0.f;
#pragma unroll
    for (int k = 0; k < kPanel; ++k)
        if (k < nm) a[(size_t)s_mv[kPanel + 1 + 2 * k] * nd + c] = y[k];
    if (c >= c0) {
#pragma unroll
        for (int j = 1; j < kPanel; ++j)
#pragma unroll
            for (int k = 0; k < j; ++k) x[j] = fmaf(-l11[j][k], x[k], x[j]);
    }
#pragma unroll
    for (int j = 0; j < kPanel; ++j)
        if (j < nb) a[(size_t)(p0 + j) * nd + c] = x[j];
}

// inverses of the diagonal blocks (kInvBlock rows) of the factors: block i,
// y = 0: the unit lower L_ii, y = 1: the upper U_ii; one thread per column of
// the inverse (forward / backward substitution on a unit vector), the block
// and the solution columns in shared memory.  Output: dinv[(2 i + y)] as a
// row-major kInvBlock x kInvBlock matrix, zero outside the block's size.
__global__ void __launch_bounds__(kInvBlock) tc_diag_inv_kernel(int nd, const float* __restrict__ a,
                                                                float* __restrict__ dinv) {
    extern __shared__ float dsh[];
    constexpr int S = kInvBlock + 1;  // padded rows
    float* blk = dsh;                  // [kInvBlock][S]
    float* y = dsh + kInvBlock * S;    // [kInvBlock][S]: y[r * S + c] = row r of column c
    pdl_wait();
    const int i = blockIdx.x, upper = blockIdx.y;
    const int r0 = i * kInvBlock, bs = min(kInvBlock, nd - r0);
    const int c = threadIdx.x;
    for (int e = c; e < kInvBlock * kInvBlock; e += blockDim.x) {
        const int r = e / kInvBlock, k = e - r * kInvBlock;
        blk[r * S + k] = (r < bs && k < bs) ? a[(size_t)(r0 + r) * nd + r0 + k] : 0.f;
        y[r * S + k] = 0.f;
    }
    __syncthreads();
    if (c < bs) {
        if (!upper) {  // L y = e_c, L unit lower
            y[c * S + c] = 1.f;
            for (int r = c + 1; r < bs; ++r) {
                float acc = 0.f;
                for (int k = c; k < r; ++k) acc = fmaf(blk[r * S + k], y[k * S + c], acc);
                y[r * S + c] = -acc;
            }
        } else {  // U y = e_c
            y[c * S + c] = __fdiv_rn(1.f, blk[c * S + c]);
            for (int r = c - 1; r >= 0; --r) {
                float acc = 0.f;
                for (int k = r + 1; k <= c; ++k) acc = fmaf(blk[r * S + k], y[k * S + c], acc);
                y[r * S + c] = __fdiv_rn(-acc, blk[r * S + r]);
            }
        }
    }
    __syncthreads();
    float* out = dinv + (size_t)(2 * i + upper) * kInvBlock * kInvBlock;
    for (int e = c; e < kInvBlock * kInvBlock; e += blockDim.x) {
        const int r = e / kInvBlock, k = e - r * kInvBlock;
        out[e] = y[r * S + k];
    }
    pdl_trigger();
}

// x = the identity (the right-hand side of the inverse's solves), perm = the identity
__global__ void tc_init_kernel(int nd, float* __restrict__ x, int* __restrict__ perm) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (long)nd * nd) {
        const int r = (int)(e / nd), c = (int)(e - (long)r * nd);
        x[e] = r == c ? 1.f : 0.f;
    }
    if (e < nd) perm[e] = (int)e;
}

// A^-1 = Z P: column perm[m] of the inverse is column m of Z = U^-1 L^-1;
// pos (the position of each original row) is perm's inverse
__global__ void tc_scatter_kernel(int nd, const float* __restrict__ z, const int* __restrict__ perm,
                                  float* __restrict__ inv, int* __restrict__ pos) {
    pdl_wait();
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)nd * nd) return;
    const int r = (int)(e / nd), m = (int)(e - (long)r * nd);
    inv[(size_t)r * nd + perm[m]] = z[e];
    if (r == 0) pos[perm[m]] = m;
}

// infinity norm (largest row sum of |a|), one warp per row; non-negative
// floats compare as their bit patterns
__global__ void tc_norm_kernel(int nd, const float* __restrict__ a, float* __restrict__ norm) {
    const long r = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= nd) return;
    float sum = 0.f;
    for (int c = lane; c < nd; c += 32) sum += fabsf(a[(size_t)r * nd + c]);
    sum = warp_sum(sum);
    if (lane == 0) atomicMax(reinterpret_cast<int*>(norm), __float_as_int(sum));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool tc_lu_supported(int nd) { return nd > 0 && nd <= kPanelRows; }

// scratch of dense_lu_inverse_tc in floats: norm, the row moves of a panel,
// perm, the diagonal inverses
constexpr int kMvInts = 64;  // >= 3 kPanel + 1
long tc_lu_scratch_floats(int nd) {
    const long nbi = (nd + kInvBlock - 1) / kInvBlock;
    return 4 + kMvInts + (long)nd + 2 * nbi * kInvBlock * kInvBlock;
}

int dense_lu_inverse_tc(int nd, float* a, int* pos, float* inv, float* x, float* work, int* err, cudaStream_t s) {
    if (nd <= 0) return BAMG_OK;
    if (!tc_lu_supported(nd)) return BAMG_EUNSUPPORTED;
    float* norm = work;
    int* mv = reinterpret_cast<int*>(work + 4);
    int* perm = mv + kMvInts;
    float* dinv = work + 4 + kMvInts + nd;
    int n = 0;
    BAMG_CUDA_TRY(cudaMemsetAsync(norm, 0, sizeof(float), s));
    tc_norm_kernel<<<(unsigned)(((long)nd * 32 + 255) / 256), 256, 0, s>>>(nd, a, norm);
    n += 1;
    tc_init_kernel<<<(unsigned)(((long)nd * nd + 255) / 256), 256, 0, s>>>(nd, x, perm);
    n += 1;
    // LU, panel by panel
    static bool attr_set = false;
    if (!attr_set) {
        BAMG_CUDA_TRY(cudaFuncSetAttribute(tc_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)panel_smem(kPanelRows)));
        BAMG_CUDA_TRY(cudaFuncSetAttribute(tc_diag_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           2 * kInvBlock * (kInvBlock + 1) * (int)sizeof(float)));
        attr_set = true;
    }
    for (int p0 = 0; p0 < nd; p0 += kPanel) {
        const int R = nd - p0, nb = min(kPanel, R), c0 = p0 + nb;
        {
            void* args[] = {&nd, &p0, &a, &mv, &perm, &norm, &err};
            if (launch_pdl((const void*)tc_panel_kernel, dim3(1), dim3(kPanelThreads), panel_smem(R), s, args) !=
                cudaSuccess)
                return BAMG_ECUDA;
        }
        {
            const int cols = nd - nb;
            if (cols > 0) {
                void* args[] = {&nd, &p0, &a, &mv};
                if (launch_pdl((const void*)tc_swap_trsm_kernel, dim3((unsigned)((cols + 255) / 256)), dim3(256), 0,
                               s, args) != cudaSuccess)
                    return BAMG_ECUDA;
                n += 1;
            }
        }
        n += 1;
        if (c0 < nd) {
            const int m = nd - c0;
            float* a22 = a + (size_t)c0 * nd + c0;
            TRY_OK(launch_tc_gemm(m, m, nb, a + (size_t)c0 * nd + p0, nd, a + (size_t)p0 * nd + c0, nd, a22, nd, a22,
                                  nd, -1.f, err, s));
        }
    }
    // inverse: blocked triangular solves on the identity, X = L^-1 (forward),
    // then Z = U^-1 X (backward); per block one product applies the diagonal
    // block's inverse to the block's rows and one updates the other blocks.
    // (Scaling the off-diagonal blocks by the diagonal inverses first saves
    // half of the launches but measured a 5x larger residual of the inverse
    // on a random 2048-unknown matrix.)
    const int nbi = (nd + kInvBlock - 1) / kInvBlock;
    {
        void* args[] = {&nd, &a, &dinv};
        if (launch_pdl((const void*)tc_diag_inv_kernel, dim3((unsigned)nbi, 2), dim3(kInvBlock),
                       2 * kInvBlock * (kInvBlock + 1) * sizeof(float), s, args) != cudaSuccess)
            return BAMG_ECUDA;
        n += 1;
    }
    for (int i = 0; i < nbi; ++i) {
        const int r0 = i * kInvBlock, bs = min(kInvBlock, nd - r0), ncol = r0 + bs;
        float* xi = x + (size_t)r0 * nd;
        // X_i = L_ii^-1 B_i (one tile row: each CTA reads its own columns of B_i before writing them)
        TRY_OK(launch_tc_gemm(bs, ncol, bs, dinv + (size_t)(2 * i) * kInvBlock * kInvBlock, kInvBlock, xi, nd,
                              nullptr, nd, xi, nd, 1.f, err, s));
        if (ncol < nd) {  // B_j -= L_ji X_i for the blocks below
            float* xb = x + (size_t)ncol * nd;
            TRY_OK(launch_tc_gemm(nd - ncol, ncol, bs, a + (size_t)ncol * nd + r0, nd, xi, nd, xb, nd, xb, nd, -1.f,
                                  err, s));
        }
    }
    for (int i = nbi - 1; i >= 0; --i) {
        const int r0 = i * kInvBlock, bs = min(kInvBlock, nd - r0);
        float* xi = x + (size_t)r0 * nd;
        TRY_OK(launch_tc_gemm(bs, nd, bs, dinv + (size_t)(2 * i + 1) * kInvBlock * kInvBlock, kInvBlock, xi, nd,
                              nullptr, nd, xi, nd, 1.f, err, s));
        if (r0 > 0)  // B_j -= U_ji Z_i for the blocks above
            TRY_OK(launch_tc_gemm(r0, nd, bs, a + r0, nd, xi, nd, x, nd, x, nd, -1.f, err, s));
    }
    {
        const float* z = x;
        void* args[] = {&nd, (void*)&z, &perm, &inv, &pos};
        if (launch_pdl((const void*)tc_scatter_kernel, dim3((unsigned)(((long)nd * nd + 255) / 256)), dim3(256), 0, s,
                       args) != cudaSuccess)
            return BAMG_ECUDA;
        n += 1;
    }
    return launched(n);
}

}  // namespace bamg
