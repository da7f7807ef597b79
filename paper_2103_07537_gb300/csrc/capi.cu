// C ABI of the bamg library: hierarchy setup, one V-cycle, FGMRES, host
// end-to-end solve, introspection.  Declarations and argument contracts are
// in include/bamg.h.  Every compute step runs in the kernels of k_*.cu; this
// file only allocates, sequences launches and reads back sizes and flags.
#include <cuda_bf16.h>
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "bamg_fields.h"
#include "common.cuh"
#include "fields.cuh"

using namespace bamg;

namespace {
std::atomic<long long> g_launches{0};
thread_local long long* t_capture_sink = nullptr;  // set while a graph is captured
}  // namespace

thread_local bool bamg::t_pdl = false;

namespace {
// programmatic dependent launch for the kernels of one V-cycle (scoped)
struct PdlScope {
    bool prev;
    explicit PdlScope(bool on) : prev(t_pdl) { t_pdl = on; }
    ~PdlScope() { t_pdl = prev; }
};
}  // namespace

// Stream-ordered device memory: one pool per device, owned by the library,
// that keeps freed memory for the next hierarchy (no cudaMalloc / cudaFree on
// the setup and destroy paths once the pool is warm).
namespace {
constexpr int kMaxDevices = 64;
std::atomic<cudaMemPool_t> g_pool[kMaxDevices];

cudaMemPool_t device_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    cudaMemPool_t p = g_pool[dev].load();
    if (p) return p;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaMemPool_t expected = nullptr;
    if (!g_pool[dev].compare_exchange_strong(expected, p)) {
        cudaMemPoolDestroy(p);
        return expected;
    }
    return p;
}

// small pinned host slots (128 bytes) for flags read back during setup and
// FGMRES, carved from process-wide blocks so that a hierarchy needs no
// cudaMallocHost of its own
std::mutex g_pin_mu;
std::vector<char*> g_pin_free;

char* pin_slot() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        char* blk = nullptr;
        if (cudaMallocHost(&blk, 64 * 128) != cudaSuccess) return nullptr;
        for (int i = 0; i < 64; ++i) g_pin_free.push_back(blk + 128 * i);
    }
    char* p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}

void pin_release(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(static_cast<char*>(p));
}

cudaError_t pool_alloc(void** q, size_t bytes, cudaStream_t s) {
    cudaMemPool_t p = device_pool();
    if (!p) return cudaMalloc(q, bytes);
    return cudaMallocFromPoolAsync(q, bytes, p, s);
}
}  // namespace

void bamg::note_launch(int count) {
    if (t_capture_sink) *t_capture_sink += count;
    else g_launches += count;
}

extern "C" long long amg_launch_count(void) { return g_launches.load(); }

namespace {

constexpr int kRapCap = 256;        // maximum stored blocks per coarse row
constexpr int kMaxCoarseDense = 4096;  // coarsest unknowns handled by the dense solve

struct Level {
    int n = 0, nnzb = 0, n_colours = 0, n_agg = 0;
    int *rp = nullptr, *ci = nullptr, *diag = nullptr;
    double* vals64 = nullptr;
    float* vals32 = nullptr;
    int *colour = nullptr, *colour_nodes = nullptr, *colour_ptr_d = nullptr;
    unsigned char* lowk = nullptr;  // per block: its column has a lower colour than its row
    int fm = 0;                     // vals32 in the field-major layout (see vrow)
    std::vector<int> colour_ptr;
    double* dinv64 = nullptr;
    float* dinv32 = nullptr;
    int *agg = nullptr, *agg_ptr = nullptr, *members = nullptr;
    void *xa = nullptr, *xb = nullptr, *xt = nullptr, *res = nullptr, *rhs = nullptr, *uc = nullptr;
    int agg_rounds = 0, colour_rounds = 0;
    // row mapping chosen for this level: smoother 0 warp per node, 1 thread per row, 2 thread per
    // row in half-size CTAs, 3 four lanes per row, 4 four lanes per row with the rows staged in
    // shared memory by asynchronous copies (steps from a zero iterate use 3), 5 four warps per
    // node, 6 / 7 sixteen / eight lanes per node taking whole blocks; residual 0 warp per row,
    // 1 thread per row
    int bgs_tpr = 0, spmv_tpr = 0;
    // measured: smoother warp / thread, residual warp / thread, smoother thread-half / split /
    // staged / wide / block-split 16 / block-split 8
    float tune_us[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    int max_row = 0;  // stored blocks in the longest row (the staged smoother's slot size)
    // persistent sweep: 0 = one launch per colour (bgs_tpr), 1 = every colour of a field step
    // in one launch (thread per row), 2 = the same with four lanes per row; the plan exists
    // when sw_tiles > 0
    int sweep = 0;
    int sw_tiles = 0;
    std::vector<int> sw_tile_ptr;  // first tile of every colour (host)
    int *sw_tile_ptr_d = nullptr, *sw_lo = nullptr, *sw_hi = nullptr;
    unsigned *sw_flags = nullptr, *sw_ctrl = nullptr;
    // measured field-step times (us): per-colour launches, sweep, sweep with four lanes per row
    float tune_step_us[3] = {0, 0, 0};
    int tune_cached = 0;  // the mappings came from an earlier tuning of the same level shape
    // ILU(0) sub-solve (sub_solver 1): factors [F][nnzb][fb][fb] in FP64 and in the cycle type,
    // elimination position of every node, higher-colour flag of every block
    double* ilu64 = nullptr;
    float* ilu32 = nullptr;
    int* pos = nullptr;
    unsigned char* upk = nullptr;
    // restricted Schwarz sub-solve (sub_solver 2): node lists of the subdomains (one per
    // aggregate), offsets of the restricted inverses of every (aggregate, field block) and
    // the inverses in FP64 and in the cycle type
    int *sd_ptr = nullptr, *sd_nodes = nullptr;
    long* sd_xoff = nullptr;
    double* sd_x64 = nullptr;
    float* sd_x32 = nullptr;
    int sd_max_m = 0;
    long sd_xtotal = 0;
    // node range of every system of a batch on this level (host and device)
    std::vector<int> sys_off;
    int* sys_off_d = nullptr;
    // fields on disjoint node sets: node range (host, device) and colour range
    // of every field, and the field of every node
    std::vector<int> fo, fcol;
    int* fo_d = nullptr;
    int* node_field = nullptr;
    // per-colour counts for the algorithmic byte / flop model (profiling only)
    std::vector<long> colour_nnz, colour_nnz_lower;
    // per-node smoother damping [n][F] (nullptr: the scalar omega) and P smoothing weights [n_agg][F]
    double* omega_s64 = nullptr;
    float* omega_s32 = nullptr;
    double* omega_p64 = nullptr;
    // smoothed prolongator of this level (F sub-blocks of fb x fb per stored block) and R = P^T
    int smoothed = 0;
    int p_nnz = 0;
    int *p_rp = nullptr, *p_ci = nullptr;
    double* p_v64 = nullptr;
    int *r_rp = nullptr, *r_i = nullptr, *r_q = nullptr;
    void *p_vc = nullptr, *r_vc = nullptr;  // P and R values in the cycle's storage type
};

struct ProfRec {
    cudaEvent_t e0, e1;
    int kind;
    double bytes, flops;
    int level;  // hierarchy level of the launch (-1: the outer Krylov method)
};
constexpr int kProfSlots = kMaxLevels + 1;  // accumulator slot = level + 1

int map_dev_error(int code) {
    switch (code) {
        case kDevOk: return BAMG_OK;
        case kDevSingularBlock: return BAMG_ESINGULAR_BLOCK;
        case kDevSingularCoarse: return BAMG_ESINGULAR_COARSE;
        case kDevBadPattern: return BAMG_EINVAL;
        case kDevRowTooLong: return BAMG_EUNSUPPORTED;
        case kDevNonFinite: return BAMG_ENAN;
        case kDevTimeout: return BAMG_ETIMEOUT;
        default: return BAMG_ECUDA;
    }
}

bool supported_block(int b, int fb) {
    switch (b * 16 + fb) {
#define CASE(BB, FF) case BB * 16 + FF:
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        return true;
        default: return false;
    }
}

}  // namespace

struct bamg_ctx {
    int b = 0, F = 1, fb = 0, nlev = 0;
    int outer_spmv_tpr = 0;  // row mapping of the FP64 outer SpMV: warp, thread, four lanes per row
    float outer_us[3] = {0, 0, 0};  // their timed launches (us; kept with the choice in the tuning cache)
    int nsys = 1;  // independent systems solved together (block-diagonal operator)
    int nf = 1;    // fields on disjoint node sets (1: co-located fields only)
    // coarsest level of a batch: one dense inverse per system
    long* inv_off_d = nullptr;
    int* row_sys_d = nullptr;
    double* binv = nullptr;
    int nd_total = 0;
    // chunks of the level-0 vectors per system (segmented reductions)
    SegTable seg{};
    // batched FGMRES workspace
    int mb_alloc = 0;
    double *bh1 = nullptr, *bh2 = nullptr, *bwsq = nullptr, *bH = nullptr, *bcs = nullptr, *bsn = nullptr,
           *bg = nullptr, *by = nullptr, *bscal = nullptr, *bsq = nullptr;
    int *bk = nullptr, *bactive = nullptr, *bincycle = nullptr;
    std::vector<double> hb_scal;
    amg_params p{};
    Level lev[kMaxLevels];
    int nd = 0;
    double *coarse_a = nullptr, *coarse_inv = nullptr;
    float* coarse_inv32 = nullptr;  // the FP32 inverse (coarse_prec 32), else null
    int* coarse_piv = nullptr;
    bool coarse_tc_used = false;  // the FP32 coarsest LU and inverse ran on the tensor cores
    long arnoldi_steps = 0, second_projections = 0;  // of the last fgmres_solve
    // fields of unequal size: the hierarchy is the padded system's (b above is
    // the padded block size); vectors are padded into pad_b / pad_x on entry
    bool padded = false;
    PadMap pad{};
    double *pad_b = nullptr, *pad_x = nullptr;
    // host-buffer entry points: the level-0 values come from host memory; their
    // copy runs on cap_stream while the setup's pattern phases run on stream,
    // and the first use of the values waits for vals_ev
    const double* vals_host = nullptr;
    cudaEvent_t vals_ev = nullptr;
    bool vals_pending = false;
    // the colouring of every level that gets a smoother runs on its own stream,
    // driven by its own host thread (its rounds poll a host flag), once the
    // hierarchy's aggregation and Galerkin products are done, beside the
    // coarsest LU and the smoother data of the other levels (it needs only the
    // level's pattern)
    struct ColourJob {
        std::thread thread;
        cudaStream_t stream = nullptr;
        cudaEvent_t ev = nullptr;
        int status = BAMG_OK, n_colours = 0, rounds = 0;
        int *flag = nullptr, *queue = nullptr, *pin = nullptr;
    } cjob[kMaxLevels];
    // the tensor-core coarsest LU enqueued on cap_stream ahead of the smoother
    // data of the finer levels (no host synchronisation inside it); its own
    // error word, its temporaries released once the setup stream has joined it
    bool coarse_pending = false;
    cudaEvent_t coarse_ev = nullptr;
    int* coarse_err = nullptr;
    std::vector<void*> coarse_tmp;
    std::vector<void*> allocs;
    long bytes = 0;
    int* d_err = nullptr;   // device error flags [4]
    int* h_pin = nullptr;   // pinned host ints [8]
    cudaStream_t cap_stream = nullptr;
    // cycle staging (graph input/output) and FP32 boundary buffers
    double *cyc_in = nullptr, *cyc_out = nullptr;
    float *r32 = nullptr, *z32 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_kernels = 0;
    // cluster tail (every level from l_tail down in one launch)
    int l_tail = -1, n_tail = 0, tail_cluster = 0;
    int tail_grid = 0;            // CTAs of the cooperative grid tail (0: cluster tail)
    unsigned* tail_bar = nullptr;  // its barrier words
    TailPhase* tail_d = nullptr;
    const void* tail_rhs = nullptr;
    const void* tail_out = nullptr;
    double tail_bytes = 0.0, tail_flops = 0.0;
    std::vector<TailPhase>* rec = nullptr;  // set while the tail phases are recorded
    double rec_bytes = 0.0, rec_flops = 0.0;
    // profiling
    int prof = 0;
    std::vector<ProfRec> recs;        // direct launches, resolved when read
    std::vector<cudaEvent_t> ev_free;
    bool capturing_prof = false;      // recording event nodes into prof_graph
    std::vector<ProfRec> graph_recs;  // event-record nodes of prof_graph
    cudaGraph_t prof_graph = nullptr;
    cudaGraphExec_t prof_exec = nullptr;
    long long prof_graph_kernels = 0;
    // resolved profile records per kernel kind and level slot
    double acc_ms[BAMG_K_COUNT][kProfSlots] = {}, acc_bytes[BAMG_K_COUNT][kProfSlots] = {},
           acc_flops[BAMG_K_COUNT][kProfSlots] = {};
    long long acc_n[BAMG_K_COUNT][kProfSlots] = {};
    int prof_level = -1;  // level of the launches being issued (profiling)
    // FGMRES workspace
    int m_alloc = 0;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *partial = nullptr, *h1 = nullptr, *h2 = nullptr,
           *wsq = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr,
           *scal = nullptr;
    unsigned* ticket = nullptr;  // last-CTA counter of the chunked reductions
    double* h_scal = nullptr;  // pinned [4]
    // host wall time of the setup phases (ms): pattern, aggregate, rap, colour, inverse, coarse, vectors,
    // learned weights
    double t_phase[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint16_t* mlp16 = nullptr;  // FP16 network parameters (learned setup)

    cudaStream_t stream = nullptr;  // the setup stream: allocations and frees are ordered on it

    // every buffer carries 64 bytes beyond its size: the asynchronous copies
    // of the staged smoother read whole 16-byte units around a row (see k_staged.cu)
    template <typename T>
    int alloc(T** ptr, size_t count) {
        *ptr = nullptr;
        if (count == 0) count = 1;
        void* q = nullptr;
        if (pool_alloc(&q, count * sizeof(T) + 64, stream) != cudaSuccess) return BAMG_ECUDA;
        allocs.push_back(q);
        bytes += (long)(count * sizeof(T));
        *ptr = static_cast<T*>(q);
        return BAMG_OK;
    }
    void release(void* q) {
        for (auto& a : allocs)
            if (a == q) {
                cudaFreeAsync(a, stream);
                a = nullptr;
            }
    }
    ~bamg_ctx() {
        for (auto& j : cjob) {
            if (j.thread.joinable()) j.thread.join();  // no kernel on memory freed below
            if (j.stream) {
                cudaStreamSynchronize(j.stream);
                cudaStreamDestroy(j.stream);
            }
            if (j.ev) cudaEventDestroy(j.ev);
            pin_release(j.pin);
        }
        if (coarse_ev) cudaEventDestroy(coarse_ev);
        if (cap_stream) cudaStreamSynchronize(cap_stream);  // no copy into memory freed below
        if (vals_ev) cudaEventDestroy(vals_ev);
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        if (prof_exec) cudaGraphExecDestroy(prof_exec);
        if (prof_graph) cudaGraphDestroy(prof_graph);
        for (auto* v : {&recs, &graph_recs})
            for (auto& r : *v) {
                cudaEventDestroy(r.e0);
                cudaEventDestroy(r.e1);
            }
        for (auto e : ev_free) cudaEventDestroy(e);
        for (void* a : allocs)
            if (a) cudaFreeAsync(a, stream);
        cudaStreamSynchronize(stream);
        pin_release(h_pin);
        pin_release(h_scal);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

#define TRY(expr)                   \
    do {                            \
        int _st = (expr);           \
        if (_st != BAMG_OK) return _st; \
    } while (0)

// ---------------------------------------------------------------------------
// dense kernels of the coarsest solve on their own
// ---------------------------------------------------------------------------
namespace {
struct DevBufs {  // device buffers freed on every return path
    std::vector<void*> p;
    ~DevBufs() {
        for (void* q : p) cudaFree(q);
    }
    template <typename T>
    int get(T** out, size_t count) {
        void* q = nullptr;
        if (cudaMalloc(&q, count * sizeof(T) + 64) != cudaSuccess) {
            (void)cudaGetLastError();
            return BAMG_ECUDA;
        }
        p.push_back(q);
        *out = static_cast<T*>(q);
        return BAMG_OK;
    }
};
int read_flag(const int* d_err, cudaStream_t s) {
    int e = 0;
    BAMG_CUDA_TRY(cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    return map_dev_error(e);
}
}  // namespace

extern "C" int amg_dense_inverse_f32(int nd, const float* a, float* inv, int method, void* stream) {
    if (nd <= 0 || !a || !inv || (method != 0 && method != 1)) return BAMG_EINVAL;
    if (method == 1 && !tc_lu_supported(nd)) return BAMG_EUNSUPPORTED;
    if ((long)nd > kMaxCoarseDense) return BAMG_EUNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBufs d;
    float *f = nullptr, *x = nullptr, *w32 = nullptr;
    int *piv = nullptr, *err = nullptr;
    double* w64 = nullptr;
    const size_t nn = (size_t)nd * nd;
    TRY(d.get(&f, nn));
    TRY(d.get(&x, nn));
    TRY(d.get(&piv, (size_t)nd));
    TRY(d.get(&err, 1));
    BAMG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    BAMG_CUDA_TRY(cudaMemcpyAsync(f, a, nn * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (method == 1) {
        TRY(d.get(&w32, (size_t)tc_lu_scratch_floats(nd)));
        TRY(dense_lu_inverse_tc(nd, f, piv, inv, x, w32, err, s));
    } else {
        TRY(d.get(&w64, (size_t)dense_lu_scratch(nd)));
        TRY(dense_lu_inverse<float>(nd, f, piv, inv, x, w64, err, s));
    }
    return read_flag(err, s);
}

extern "C" int amg_gemm_tc_f32(int m, int n, int k, const float* A, int lda, const float* B, int ldb, float* C,
                               int ldc, void* stream) {
    if (m < 0 || n < 0 || k < 0 || lda < k || ldb < n || ldc < n || (m > 0 && n > 0 && (!C || (k > 0 && (!A || !B)))))
        return BAMG_EINVAL;
    if (m == 0 || n == 0) return BAMG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBufs d;
    int* err = nullptr;
    TRY(d.get(&err, 1));
    BAMG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    TRY(launch_tc_gemm(m, n, k, A, lda, B, ldb, C, ldc, C, ldc, 1.f, err, s));
    return read_flag(err, s);
}


// read the device error flags (synchronises s)
static int check_dev(bamg_ctx* h, cudaStream_t s) {
    BAMG_CUDA_TRY(cudaMemcpyAsync(h->h_pin, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    return map_dev_error(h->h_pin[0]);
}

// ---------------------------------------------------------------------------
// per-launch event timing (only while profiling is enabled)
// ---------------------------------------------------------------------------
static cudaEvent_t take_event(bamg_ctx* h) {
    if (!h->ev_free.empty()) {
        cudaEvent_t e = h->ev_free.back();
        h->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// While a profiling graph is captured the events become event-record nodes of
// the graph (timestamps taken by the GPU between the kernels, no host gaps).
static int prof_begin(bamg_ctx* h, cudaStream_t s) {
    if (!h->prof) return -1;
    ProfRec r{take_event(h), take_event(h), -1, 0.0, 0.0, h->prof_level};
    std::vector<ProfRec>& v = h->capturing_prof ? h->graph_recs : h->recs;
    if (h->capturing_prof) cudaEventRecordWithFlags(r.e0, s, cudaEventRecordExternal);
    else cudaEventRecord(r.e0, s);
    v.push_back(r);
    return (int)v.size() - 1;
}

static void prof_end(bamg_ctx* h, cudaStream_t s, int idx, int kind, double bytes, double flops) {
    if (idx < 0) return;
    ProfRec& r = (h->capturing_prof ? h->graph_recs : h->recs)[(size_t)idx];
    if (h->capturing_prof) cudaEventRecordWithFlags(r.e1, s, cudaEventRecordExternal);
    else cudaEventRecord(r.e1, s);
    r.kind = kind;
    r.bytes = bytes;
    r.flops = flops;
}

// launch with optional timing: needs h and s in scope
#define PL(kind, bytes, flops, expr)                     \
    do {                                                 \
        const int _pi = prof_begin(h, s);                \
        const int _st = (expr);                          \
        prof_end(h, s, _pi, (kind), (bytes), (flops));   \
        if (_st != BAMG_OK) return _st;                  \
    } while (0)

extern "C" void amg_default_params(amg_params* p) {
    if (!p) return;
    p->max_levels = 10;
    p->max_coarse = 2500;
    p->n_pre = 1;
    p->n_post = 1;
    p->omega = 0.5;
    p->cycle_prec = 64;
    p->use_graph = 1;
    p->tail_dofs = 0;
    p->autotune = 1;
    p->smooth_p = 0;
    p->omega_p = 0.0;
    p->omega_s_arr = nullptr;
    p->omega_s_len = 0;
    p->omega_p_arr = nullptr;
    p->omega_p_len = 0;
    p->mlp = nullptr;
    p->pr_storage = 32;
    p->mlp_levels = 0;
    p->use_pdl = 1;
    p->coarse_prec = 64;
    p->tail_grid = 0;
    p->value_layout = 0;
    p->sweep = 0;
    p->sub_solver = 0;
    p->schwarz_overlap = 1;
    p->ortho = 0;
    p->coarse_tc = 1;
    p->inner_sweeps = 1;
}

extern "C" const char* amg_strerror(int status) {
    switch (status) {
        case BAMG_OK: return "ok";
        case BAMG_NOT_CONVERGED: return "not converged within max_iter";
        case BAMG_EINVAL: return "invalid argument or matrix pattern";
        case BAMG_ECUDA: return "CUDA runtime error";
        case BAMG_ESINGULAR_BLOCK: return "singular node diagonal block";
        case BAMG_ESINGULAR_COARSE: return "singular coarsest operator";
        case BAMG_ENAN: return "non-finite value";
        case BAMG_ETIMEOUT: return "setup iteration bound exceeded";
        case BAMG_EUNSUPPORTED: return "size or block shape not supported";
        default: return "unknown status";
    }
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
static int setup_tail(bamg_ctx* h, cudaStream_t s);
static int record_tail(bamg_ctx* h, cudaStream_t s, bool only_counts);

using Clock = std::chrono::steady_clock;
static double ms_since(Clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

template <typename T>
static const T* level_vals(const Level& L);
// layout flag of level_vals<T>: the FP64 values are always block-major
template <typename T>
static int level_fm(const Level& L) {
    return sizeof(T) == 4 ? L.fm : 0;
}
template <>
const double* level_vals<double>(const Level& L) { return L.vals64; }
template <>
const float* level_vals<float>(const Level& L) { return L.vals32; }
template <typename T>
static const T* level_ilu(const Level& L);
template <>
const double* level_ilu<double>(const Level& L) { return L.ilu64; }
template <>
const float* level_ilu<float>(const Level& L) { return L.ilu32; }
template <typename T>
static const T* level_dinv(const Level& L);
template <>
const double* level_dinv<double>(const Level& L) { return L.dinv64; }
template <>
const float* level_dinv<float>(const Level& L) { return L.dinv32; }
template <typename T>
static const T* level_omega(const Level& L);
template <>
const double* level_omega<double>(const Level& L) { return L.omega_s64; }
template <>
const float* level_omega<float>(const Level& L) { return L.omega_s32; }

// The damping weights of level l, which is being coarsened (its aggregates
// and member lists exist): from the network on the level's features, from
// the caller's per-level arrays, or the constants.  Sets L.smoothed.
static int level_weights(bamg_ctx* h, int l, cudaStream_t s, long long* used_s, long long* used_p) {
    Level& L = h->lev[l];
    const amg_params& p = h->p;
    const int F = h->F;
    const size_t ns = (size_t)L.n * F, np = (size_t)L.n_agg * F;
    if (p.mlp && p.mlp_levels > 0 && l >= p.mlp_levels) {  // beyond the network's depths: plain
        L.smoothed = 0;
        return BAMG_OK;
    }
    if (p.mlp) {
        float *nf = nullptr, *af = nullptr, *yn = nullptr, *ya = nullptr;
        int* cnt = nullptr;
        TRY(h->alloc(&nf, ns * BAMG_NFEAT));
        TRY(h->alloc(&af, np * BAMG_NFEAT));
        TRY(h->alloc(&yn, ns * BAMG_MLP_OUT));
        TRY(h->alloc(&ya, np * BAMG_MLP_OUT));
        TRY(h->alloc(&cnt, (size_t)L.n_agg + 1));
        TRY(h->alloc(&L.omega_s64, ns));
        TRY(h->alloc(&L.omega_p64, np));
        TRY(launch_agg_count(L.n, L.n_agg, L.agg, cnt, h->d_err, s));
        TRY(launch_features(h->b, h->fb, L.n, L.rp, L.ci, L.vals64, L.agg, cnt, l, nf, h->d_err, s));
        TRY(launch_agg_features(L.n_agg, F, L.agg_ptr, L.members, nf, af, s));
        TRY(launch_mlp_forward(h->mlp16, nf, (int)ns, yn, s));
        TRY(launch_mlp_forward(h->mlp16, af, (int)np, ya, s));
        BAMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int), s));
        TRY(launch_omega_from_mlp((int)ns, 0, yn, L.omega_s64, nullptr, s));
        TRY(launch_omega_from_mlp((int)np, 1, ya, L.omega_p64, cnt, s));
        BAMG_CUDA_TRY(cudaMemcpyAsync(h->h_pin + 4, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
        TRY(check_dev(h, s));
        L.smoothed = h->h_pin[4] != 0;  // P smoothed only where a weight survived the clip
        for (void* q : {(void*)nf, (void*)af, (void*)yn, (void*)ya, (void*)cnt}) h->release(q);
        return BAMG_OK;
    }
    if (p.omega_s_arr) {
        if (*used_s + (long long)ns > p.omega_s_len) return BAMG_EINVAL;
        TRY(h->alloc(&L.omega_s64, ns));
        BAMG_CUDA_TRY(cudaMemcpyAsync(L.omega_s64, p.omega_s_arr + *used_s, sizeof(double) * ns,
                                      cudaMemcpyHostToDevice, s));
        *used_s += (long long)ns;
    }
    L.smoothed = p.smooth_p;
    if (p.smooth_p) {
        TRY(h->alloc(&L.omega_p64, np));
        if (p.omega_p_arr) {
            if (*used_p + (long long)np > p.omega_p_len) return BAMG_EINVAL;
            BAMG_CUDA_TRY(cudaMemcpyAsync(L.omega_p64, p.omega_p_arr + *used_p, sizeof(double) * np,
                                          cudaMemcpyHostToDevice, s));
            *used_p += (long long)np;
        } else {
            TRY(launch_fill((long)np, p.omega_p, L.omega_p64, s));
        }
    }
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));  // the host arrays are the caller's
    return BAMG_OK;
}

// rows, columns of a row-wise product into (rp, ci): symbolic pass, scan, fill
static int product_pattern(bamg_ctx* h, int nrows, const int* xrp, const int* xci, const int* xmap, const int* yrp,
                           const int* yci, int** rp_out, int** ci_out, int* nnz_out, cudaStream_t s) {
    int *count = nullptr, *tmp_cols = nullptr, *scan = nullptr;
    TRY(h->alloc(&count, (size_t)nrows + 1));
    TRY(h->alloc(&tmp_cols, (size_t)nrows * kRapCap));
    TRY(h->alloc(&scan, (size_t)scan_tmp_bytes(nrows) / sizeof(int) + 16));
    TRY(h->alloc(rp_out, (size_t)nrows + 1));
    TRY(spgemm_symbolic(nrows, xrp, xci, xmap, yrp, yci, count, tmp_cols, kRapCap, h->d_err, s));
    TRY(check_dev(h, s));
    TRY(exclusive_scan(nrows, count, *rp_out, scan, scan_tmp_bytes(nrows) + 64, s));
    BAMG_CUDA_TRY(cudaMemcpyAsync(h->h_pin, *rp_out + nrows, sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    *nnz_out = h->h_pin[0];
    TRY(h->alloc(ci_out, (size_t)*nnz_out));
    TRY(rap_fill_cols(nrows, *rp_out, tmp_cols, kRapCap, *ci_out, s));
    h->release(count);
    h->release(tmp_cols);
    h->release(scan);
    return BAMG_OK;
}

// Smoothed prolongator of level l, R = P^T, and A_{l+1} = R (A_l P).
static int smoothed_galerkin(bamg_ctx* h, int l, cudaStream_t s) {
    Level& L = h->lev[l];
    Level& C = h->lev[l + 1];
    const int b = h->b, F = h->F, fb = h->fb, n = L.n, nc = L.n_agg;
    if (!L.dinv64) {
        TRY(h->alloc(&L.dinv64, (size_t)n * F * fb * fb));
        TRY(block_inverses(b, fb, n, L.diag, L.vals64, L.dinv64, h->d_err, s));
        TRY(check_dev(h, s));
    }
    // P: row i holds the distinct agg(j) of its stored j
    TRY(product_pattern(h, n, L.rp, L.ci, L.agg, nullptr, nullptr, &L.p_rp, &L.p_ci, &L.p_nnz, s));
    TRY(h->alloc(&L.p_v64, (size_t)L.p_nnz * F * fb * fb));
    TRY(prolongator_numeric(b, fb, n, L.rp, L.ci, L.vals64, L.dinv64, L.agg, L.omega_p64, L.p_rp, L.p_ci, L.p_v64,
                            s));
    // R = P^T: coarse row I holds the neighbours of I's members, ascending
    int nnz_r = 0;
    TRY(product_pattern(h, nc, L.agg_ptr, L.members, nullptr, L.rp, L.ci, &L.r_rp, &L.r_i, &nnz_r, s));
    if (nnz_r != L.p_nnz) return BAMG_ECUDA;
    TRY(h->alloc(&L.r_q, (size_t)nnz_r));
    TRY(transpose_index(nc, L.r_rp, L.r_i, L.p_rp, L.p_ci, L.r_q, h->d_err, s));
    // A P, then R (A P)
    int *ap_rp = nullptr, *ap_ci = nullptr, nnz_ap = 0;
    TRY(product_pattern(h, n, L.rp, L.ci, nullptr, L.p_rp, L.p_ci, &ap_rp, &ap_ci, &nnz_ap, s));
    double* ap_v = nullptr;
    TRY(h->alloc(&ap_v, (size_t)nnz_ap * b * b));
    TRY(ap_numeric(b, fb, n, L.rp, L.ci, L.vals64, L.p_rp, L.p_ci, L.p_v64, ap_rp, ap_ci, ap_v, s));
    C.n = nc;
    TRY(product_pattern(h, nc, L.r_rp, L.r_i, nullptr, ap_rp, ap_ci, &C.rp, &C.ci, &C.nnzb, s));
    TRY(h->alloc(&C.vals64, (size_t)C.nnzb * b * b));
    TRY(rap_general_numeric(b, fb, nc, L.r_rp, L.r_i, L.r_q, L.p_v64, ap_rp, ap_ci, ap_v, C.rp, C.ci, C.vals64, s));
    TRY(check_dev(h, s));
    h->release(ap_rp);
    h->release(ap_ci);
    h->release(ap_v);
    // transfer values in the cycle's storage type
    const long nnz = L.p_nnz;
    const size_t m = (size_t)nnz * F * fb * fb;
    if (h->p.cycle_prec == 64) {
        double *pv = nullptr, *rv = nullptr;
        TRY(h->alloc(&pv, m));
        TRY(h->alloc(&rv, m));
        TRY(transfer_values<double>(nnz, F, fb, L.r_q, L.p_v64, pv, rv, s));
        L.p_vc = pv;
        L.r_vc = rv;
    } else if (h->p.pr_storage == 16) {
        __nv_bfloat16 *pv = nullptr, *rv = nullptr;
        TRY(h->alloc(&pv, m));
        TRY(h->alloc(&rv, m));
        TRY(transfer_values<__nv_bfloat16>(nnz, F, fb, L.r_q, L.p_v64, pv, rv, s));
        L.p_vc = pv;
        L.r_vc = rv;
    } else {
        float *pv = nullptr, *rv = nullptr;
        TRY(h->alloc(&pv, m));
        TRY(h->alloc(&rv, m));
        TRY(transfer_values<float>(nnz, F, fb, L.r_q, L.p_v64, pv, rv, s));
        L.p_vc = pv;
        L.r_vc = rv;
    }
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    return BAMG_OK;
}

// Subdomains of the restricted Schwarz sub-solve on level l (its aggregates
// extended by schwarz_overlap layers in the graph of A_ff) and the own rows of
// their local inverses (FP64, and in the cycle type for FP32 cycles).
static int schwarz_level(bamg_ctx* h, int l, cudaStream_t s) {
    Level& L = h->lev[l];
    const int na = L.n_agg, fb = h->fb;
    const int nfs = h->nf > 1 ? 1 : h->F;  // subdomains per aggregate
    const int* nfield = h->nf > 1 ? L.node_field : nullptr;
    int* cnt = nullptr;
    TRY(h->alloc(&cnt, (size_t)na));
    TRY(schwarz_setup_count(na, L.agg_ptr, L.members, L.rp, L.ci, nfield, h->p.schwarz_overlap, cnt, s));
    std::vector<int> c((size_t)na), ap((size_t)na + 1);
    BAMG_CUDA_TRY(cudaMemcpyAsync(c.data(), cnt, sizeof(int) * na, cudaMemcpyDeviceToHost, s));
    BAMG_CUDA_TRY(cudaMemcpyAsync(ap.data(), L.agg_ptr, sizeof(int) * (na + 1), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    h->release(cnt);
    std::vector<int> sp((size_t)na + 1, 0);
    std::vector<long> xo((size_t)na * nfs + 1, 0);
    int max_m = 0;
    for (int I = 0; I < na; ++I) {
        if (c[I] < 0) return BAMG_EUNSUPPORTED;  // a subdomain larger than the local solve takes
        sp[I + 1] = sp[I] + c[I];
        const int m = c[I] * fb;
        max_m = m > max_m ? m : max_m;
        const long own = (long)(ap[I + 1] - ap[I]) * fb;
        for (int f = 0; f < nfs; ++f) xo[(size_t)I * nfs + f + 1] = xo[(size_t)I * nfs + f] + own * m;
    }
    L.sd_max_m = max_m;
    L.sd_xtotal = xo.back();
    TRY(h->alloc(&L.sd_ptr, (size_t)na + 1));
    TRY(h->alloc(&L.sd_nodes, (size_t)sp.back()));
    TRY(h->alloc(&L.sd_xoff, xo.size()));
    TRY(h->alloc(&L.sd_x64, (size_t)L.sd_xtotal));
    BAMG_CUDA_TRY(cudaMemcpyAsync(L.sd_ptr, sp.data(), sizeof(int) * sp.size(), cudaMemcpyHostToDevice, s));
    BAMG_CUDA_TRY(cudaMemcpyAsync(L.sd_xoff, xo.data(), sizeof(long) * xo.size(), cudaMemcpyHostToDevice, s));
    TRY(schwarz_setup_fill(na, nfs, h->b, fb, max_m, L.agg_ptr, L.members, L.rp, L.ci, nfield,
                           h->p.schwarz_overlap, L.sd_ptr, L.sd_nodes, L.vals64, L.sd_xoff, L.sd_x64, h->d_err, s));
    TRY(check_dev(h, s));
    if (h->p.cycle_prec == 32) {
        TRY(h->alloc(&L.sd_x32, (size_t)L.sd_xtotal));
        TRY(launch_convert_d2f(L.sd_xtotal, L.sd_x64, L.sd_x32, s));
    }
    return BAMG_OK;
}

// Tiles of the persistent sweep on a coloured level (colour lists and lowk
// exist) and their dependencies; skipped when sweeps are off, for sub-block
// sizes without a sweep kernel and for levels with more colours than it takes.
static int build_sweep_plan(bamg_ctx* h, Level& L, cudaStream_t s) {
    const int ntile = sweep_tile_nodes(h->fb);
    if (h->p.sweep == 1 || ntile <= 0 || L.n_colours < 1 || L.n_colours > kSweepMaxColours) return BAMG_OK;
    const int C = L.n_colours;
    L.sw_tile_ptr.assign((size_t)C + 1, 0);
    for (int c = 0; c < C; ++c)
        L.sw_tile_ptr[c + 1] = L.sw_tile_ptr[c] + ceil_div(L.colour_ptr[c + 1] - L.colour_ptr[c], ntile);
    L.sw_tiles = L.sw_tile_ptr[C];
    TRY(h->alloc(&L.sw_tile_ptr_d, (size_t)C + 1));
    TRY(h->alloc(&L.sw_lo, (size_t)L.sw_tiles * C));
    TRY(h->alloc(&L.sw_hi, (size_t)L.sw_tiles * C));
    TRY(h->alloc(&L.sw_flags, (size_t)L.sw_tiles));
    TRY(h->alloc(&L.sw_ctrl, 4));
    int* tile_of = nullptr;
    TRY(h->alloc(&tile_of, (size_t)L.n));
    BAMG_CUDA_TRY(cudaMemcpyAsync(L.sw_tile_ptr_d, L.sw_tile_ptr.data(), sizeof(int) * (C + 1), cudaMemcpyHostToDevice,
                                  s));
    BAMG_CUDA_TRY(cudaMemsetAsync(L.sw_flags, 0, sizeof(unsigned) * (size_t)L.sw_tiles, s));
    BAMG_CUDA_TRY(cudaMemsetAsync(L.sw_ctrl, 0, 4 * sizeof(unsigned), s));
    TRY(sweep_plan(L.n, C, ntile, L.colour_nodes, L.colour, L.colour_ptr_d, L.sw_tile_ptr_d, L.rp, L.ci, L.lowk,
                   L.sw_tiles, tile_of, L.sw_lo, L.sw_hi, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    h->release(tile_of);
    if (h->p.sweep >= 2) L.sweep = h->p.sweep - 1;
    return BAMG_OK;
}

// the sweep arguments of colours c_lo..c_hi-1 of level L
static SweepArgs sweep_args(bamg_ctx* h, const Level& L, int c_lo, int c_hi) {
    SweepArgs sw;
    sw.c_lo = c_lo;
    sw.c_hi = c_hi;
    sw.C = L.n_colours;
    sw.colour_ptr = L.colour_ptr_d;
    sw.tile_ptr = L.sw_tile_ptr_d;
    sw.dep_lo = L.sw_lo;
    sw.dep_hi = L.sw_hi;
    sw.flags = L.sw_flags;
    sw.ctrl = L.sw_ctrl;
    sw.err = h->d_err;
    return sw;
}

// one colour of a field step in the level's row mapping (the staged kernel
// for steps that read whole rows; from a zero iterate its four-lanes twin,
// which gives the same values)
template <typename T>
static int launch_colour_step(bamg_ctx* h, const Level& L, const BgsArgs& a, cudaStream_t s) {
    if (L.bgs_tpr == 6 || L.bgs_tpr == 7)
        return launch_bgs_colour_bsp<T>(h->b, h->fb, a, L.bgs_tpr == 6 ? 16 : 8, s);
    if (L.bgs_tpr == 5) return launch_bgs_colour_wide<T>(h->b, h->fb, a, s);
    if (L.bgs_tpr == 4 && a.x_in) return launch_bgs_colour_staged<T>(h->b, h->fb, a, L.max_row, h->d_err, s);
    if (L.bgs_tpr == 4) return launch_bgs_colour_tpr<T>(h->b, h->fb, a, s, 2);
    return L.bgs_tpr ? launch_bgs_colour_tpr<T>(h->b, h->fb, a, s, L.bgs_tpr - 1)
                     : launch_bgs_colour<T>(h->b, h->fb, a, s);
}

// a non-default row mapping must beat warp-per-row by more than 3%
constexpr float kTuneMargin = 0.97f;

// average device time (us) of `reps` launches of f after one warm-up launch
template <class F>
static float time_launch(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps, F&& f) {
    if (f() != BAMG_OK) return 1e30f;
    auto timed = [&](int n) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < n; ++r)
            if (f() != BAMG_OK) return 1e30f;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return 1e3f * ms / n;
    };
    // launches of 40 us and more are timed over 3 (their noise is small
    // against the tuning margin); shorter ones over reps
    const float first = timed(3);
    return first >= 40.0f ? first : timed(reps);
}

// Decisions of the autotuner, kept per process for every level shape they
// were measured on: a later setup of a level with the same shape (the same
// pattern again, as in a sequence of Newton or time steps) takes the
// recorded mappings instead of timing the launches again.  Only the choice
// of kernels is kept, never a value.  The key holds everything the choice
// depends on: device, sizes of the level and of every colour, block shape,
// fields, precision, value layout, launch mode and sub-solver.
struct TuneRec {
    int bgs_tpr, spmv_tpr, sweep;
    float tune_us[10], tune_step_us[3];
};
std::mutex g_tune_mu;
std::vector<std::pair<std::string, TuneRec>> g_tune;  // small: one entry per distinct level shape
struct OuterRec {
    int mapping;
    float us[3];
};
std::vector<std::pair<std::string, OuterRec>> g_tune_outer;  // outer FP64 SpMV mapping per level-0 shape

static std::string tune_key(const bamg_ctx* h, const Level& L, int l) {
    int dev = -1;
    cudaGetDevice(&dev);
    std::string k = std::to_string(dev) + "/" + std::to_string(l) + "/" + std::to_string(L.n) + "/" +
                    std::to_string(L.nnzb) + "/" + std::to_string(h->b) + "/" + std::to_string(h->fb) + "/" +
                    std::to_string(h->nf) + "/" + std::to_string(h->nsys) + "/" + std::to_string(h->p.cycle_prec) +
                    "/" + std::to_string(L.fm) + "/" + std::to_string(h->p.use_pdl) + "/" +
                    std::to_string(h->p.sub_solver) + "/" + std::to_string(h->p.sweep) + "/" +
                    std::to_string(L.sw_tiles) + "/" +
                    std::to_string(L.omega_s64 != nullptr) + "/";
    for (int c = 0; c <= L.n_colours; ++c) k += std::to_string(L.colour_ptr[c]) + ",";
    return k;
}

// Autotuner: per level, time the row mappings of the smoother (first colour,
// first field) and of the residual SpMV on the level's own operator, and keep
// the faster; likewise for the FP64 outer SpMV.  (Timing whole sweeps instead
// doubled the setup of the 2D workload and picked no better mappings.)
template <typename T>
static int autotune_levels(bamg_ctx* h, cudaStream_t s) {
    cudaEvent_t e0, e1;
    BAMG_CUDA_TRY(cudaEventCreate(&e0));
    BAMG_CUDA_TRY(cudaEventCreate(&e1));
    const int b = h->b;
    for (int l = 0; l + 1 < h->nlev; ++l) {
        Level& L = h->lev[l];
        const std::string key = h->p.autotune == 1 ? tune_key(h, L, l) : std::string();
        if (h->p.autotune == 1) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            bool hit = false;
            for (const auto& e : g_tune)
                if (e.first == key) {
                    L.bgs_tpr = e.second.bgs_tpr;
                    L.spmv_tpr = e.second.spmv_tpr;
                    L.sweep = e.second.sweep;
                    memcpy(L.tune_us, e.second.tune_us, sizeof L.tune_us);
                    memcpy(L.tune_step_us, e.second.tune_step_us, sizeof L.tune_step_us);
                    hit = true;
                    break;
                }
            if (hit) {
                L.tune_cached = 1;
                continue;
            }
        }
        const size_t nb = (size_t)L.n * b;
        BAMG_CUDA_TRY(cudaMemsetAsync(L.xa, 0, nb * sizeof(T), s));
        BAMG_CUDA_TRY(cudaMemsetAsync(L.res, 0, nb * sizeof(T), s));
        BAMG_CUDA_TRY(cudaMemsetAsync(L.xt, 0, (size_t)L.n * h->fb * sizeof(T), s));
        BgsArgs a;
        a.n_in_colour = L.colour_ptr[1] - L.colour_ptr[0];
        a.nodes = L.colour_nodes;
        a.colour = 0;
        a.colours = L.colour;
        a.lowk = L.lowk;
        a.fm = level_fm<T>(L);
        a.rp = L.rp;
        a.ci = L.ci;
        a.vals = level_vals<T>(L);
        a.dinv = level_dinv<T>(L);
        a.rhs = L.res;
        a.x_in = L.xa;
        a.x_out = L.xb;
        a.xt = L.xt;
        a.uc = nullptr;
        a.agg = nullptr;
        a.field = 0;
        a.F = h->F;
        a.omega = h->p.omega;
        a.omega_node = level_omega<T>(L);
        // 10 timed launches per candidate; a thread-per-row mapping replaces the
        // warp-per-row one only when it is faster by more than kTuneMargin (3
        // launches and a plain minimum flipped between runs on near ties)
        const int reps = 10;
        L.tune_us[0] = time_launch(s, e0, e1, reps, [&] { return launch_bgs_colour<T>(b, h->fb, a, s); });
        L.tune_us[1] = time_launch(s, e0, e1, reps, [&] { return launch_bgs_colour_tpr<T>(b, h->fb, a, s, 0); });
        L.tune_us[4] = time_launch(s, e0, e1, reps, [&] { return launch_bgs_colour_tpr<T>(b, h->fb, a, s, 1); });
        L.tune_us[5] = time_launch(s, e0, e1, reps, [&] { return launch_bgs_colour_tpr<T>(b, h->fb, a, s, 2); });
        L.tune_us[6] = time_launch(s, e0, e1, reps,
                                   [&] { return launch_bgs_colour_staged<T>(b, h->fb, a, L.max_row, h->d_err, s); });
        L.tune_us[7] = time_launch(s, e0, e1, reps, [&] { return launch_bgs_colour_wide<T>(b, h->fb, a, s); });
        L.tune_us[8] = time_launch(s, e0, e1, reps, [&] { return launch_bgs_colour_bsp<T>(b, h->fb, a, 16, s); });
        L.tune_us[9] = time_launch(s, e0, e1, reps, [&] { return launch_bgs_colour_bsp<T>(b, h->fb, a, 8, s); });
        const T* x = static_cast<const T*>(L.xa);
        const T* r = static_cast<const T*>(L.res);
        T* y = static_cast<T*>(L.xb);
        L.tune_us[2] = time_launch(s, e0, e1, reps,
                                   [&] {
                                       return launch_spmv<T>(b, h->fb, level_fm<T>(L), L.n, L.rp, L.ci,
                                                             level_vals<T>(L), x, r, y, s);
                                   });
        L.tune_us[3] = time_launch(
            s, e0, e1, reps,
            [&] {
                return launch_spmv_tpr<T>(b, h->fb, level_fm<T>(L), L.n, L.rp, L.ci, level_vals<T>(L), x, r, y, s);
            });
        if (h->p.autotune >= 2) L.bgs_tpr = h->p.autotune - 1;
        else if (h->p.autotune == 1) {
            // the fastest thread-per-row variant replaces warp per node only by the margin
            const float tv[7] = {L.tune_us[1], L.tune_us[4], L.tune_us[5], L.tune_us[6],
                                 L.tune_us[7], L.tune_us[8], L.tune_us[9]};
            int best = 0;
            for (int v = 1; v < 7; ++v)
                if (tv[v] < tv[best]) best = v;
            // (four warps per node replaces one warp per node on any win: the
            // same per-node structure, and in the cycle, with programmatic
            // dependent launches, it gained 7% on the 3D level 1 where the
            // isolated timing saw 0.6-3%)
            L.bgs_tpr = tv[best] < (best == 4 ? 1.0f : kTuneMargin) * L.tune_us[0] ? best + 1 : 0;
        }
        if (L.bgs_tpr == 4 && L.tune_us[6] >= 1e29f) L.bgs_tpr = 3;  // the staged kernel does not take this level
        if ((L.bgs_tpr == 6 || L.bgs_tpr == 7) && !bsp_supported(b, h->fb)) L.bgs_tpr = 3;  // block too large
        if (h->p.autotune == 1 && h->p.use_pdl && (L.bgs_tpr == 0 || L.bgs_tpr == 5)) {
            // warp against four warps per node again, as a whole field step
            // (every colour of field 0) in the cycle's launch mode: with
            // programmatic dependent launches each kernel's loads before its
            // wait overlap the previous colour, which favours the wider mapping
            // (3D level 1: 7% faster in the cycle, within 3% one colour alone)
            PdlScope pdl(true);
            const int c_hi = h->nf > 1 ? L.fcol[1] : L.n_colours;
            float tstep[2] = {0.f, 0.f};
            for (int m = 0; m < 2; ++m) {
                L.bgs_tpr = m == 0 ? 0 : 5;
                tstep[m] = time_launch(s, e0, e1, reps, [&]() {
                    for (int c = 0; c < c_hi; ++c) {
                        BgsArgs ac = a;
                        ac.n_in_colour = L.colour_ptr[c + 1] - L.colour_ptr[c];
                        ac.nodes = L.colour_nodes + L.colour_ptr[c];
                        ac.colour = c;
                        const int st = launch_colour_step<T>(h, L, ac, s);
                        if (st != BAMG_OK) return st;
                    }
                    return (int)BAMG_OK;
                });
            }
            L.bgs_tpr = tstep[1] < tstep[0] ? 5 : 0;
        }
        L.spmv_tpr = h->p.autotune >= 2 || (h->p.autotune == 1 && L.tune_us[3] < kTuneMargin * L.tune_us[2]);
        // one whole field step (every colour of field 0) as per-colour launches
        // in the chosen mapping against the persistent sweep, in the cycle's
        // launch mode; the sweep replaces the per-colour launches by the margin
        if (L.sw_tiles > 0 && h->p.sweep == 0 && h->p.autotune == 1) {
            PdlScope pdl(h->p.use_pdl != 0);
            const int c_hi = h->nf > 1 ? L.fcol[1] : L.n_colours;
            auto per_colour = [&]() {
                for (int c = 0; c < c_hi; ++c) {
                    BgsArgs ac = a;
                    ac.n_in_colour = L.colour_ptr[c + 1] - L.colour_ptr[c];
                    ac.nodes = L.colour_nodes + L.colour_ptr[c];
                    ac.colour = c;
                    const int st = launch_colour_step<T>(h, L, ac, s);
                    if (st != BAMG_OK) return st;
                }
                return (int)BAMG_OK;
            };
            const SweepArgs sw = sweep_args(h, L, 0, c_hi);
            const int tiles = L.sw_tile_ptr[c_hi];
            L.tune_step_us[0] = time_launch(s, e0, e1, reps, per_colour);
            L.tune_step_us[1] = time_launch(s, e0, e1, reps, [&] {
                return launch_bgs_sweep<T>(b, h->fb, a, sw, tiles, 0, s);
            });
            L.tune_step_us[2] = time_launch(s, e0, e1, reps, [&] {
                return launch_bgs_sweep<T>(b, h->fb, a, sw, tiles, 1, s);
            });
            const int best = L.tune_step_us[2] < L.tune_step_us[1] ? 2 : 1;
            L.sweep = L.tune_step_us[best] < kTuneMargin * L.tune_step_us[0] ? best : 0;
            TRY(check_dev(h, s));
        }
        if (h->p.autotune == 1) {
            TuneRec rec;
            rec.bgs_tpr = L.bgs_tpr;
            rec.spmv_tpr = L.spmv_tpr;
            rec.sweep = L.sweep;
            memcpy(rec.tune_us, L.tune_us, sizeof rec.tune_us);
            memcpy(rec.tune_step_us, L.tune_step_us, sizeof rec.tune_step_us);
            std::lock_guard<std::mutex> lk(g_tune_mu);
            if (g_tune.size() < 4096) g_tune.emplace_back(key, rec);
        }
    }
    int outer_cached = -1;
    std::string okey;
    if (h->p.autotune == 1) {
        int dev = -1;
        cudaGetDevice(&dev);
        const Level& L0 = h->lev[0];
        okey = std::to_string(dev) + "/" + std::to_string(L0.n) + "/" + std::to_string(L0.nnzb) + "/" +
               std::to_string(b) + "/" + std::to_string(h->nsys);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto& e : g_tune_outer)
            if (e.first == okey) {
                outer_cached = e.second.mapping;
                memcpy(h->outer_us, e.second.us, sizeof h->outer_us);
            }
    }
    if (outer_cached >= 0) {
        h->outer_spmv_tpr = outer_cached;
    } else {
        const Level& L0 = h->lev[0];
        BAMG_CUDA_TRY(cudaMemsetAsync(h->cyc_in, 0, sizeof(double) * (size_t)L0.n * b, s));
        const float t0 = time_launch(s, e0, e1, 10, [&] {
            return launch_spmv<double>(b, h->fb, 0, L0.n, L0.rp, L0.ci, L0.vals64, h->cyc_in, nullptr, h->cyc_out, s);
        });
        const float t1 = time_launch(s, e0, e1, 10, [&] {
            return launch_spmv_tpr<double>(b, h->fb, 0, L0.n, L0.rp, L0.ci, L0.vals64, h->cyc_in, nullptr, h->cyc_out,
                                           s);
        });
        const float t2 = time_launch(s, e0, e1, 10, [&] {
            return launch_spmv_tpr<double>(b, h->fb, 0, L0.n, L0.rp, L0.ci, L0.vals64, h->cyc_in, nullptr, h->cyc_out,
                                           s, 1);
        });
        h->outer_us[0] = t0;
        h->outer_us[1] = t1;
        h->outer_us[2] = t2;
        // 0 warp per row, 1 thread per row, 2 four lanes per row: a thread mapping
        // replaces warp per row by the margin
        const float tt[2] = {t1, t2};
        const int bt = t2 < t1 ? 1 : 0;
        h->outer_spmv_tpr = h->p.autotune >= 2 ? (h->p.autotune == 4 || h->p.autotune == 5 ? 2 : 1)
                            : (h->p.autotune == 1 && tt[bt] < kTuneMargin * t0) ? bt + 1
                                                                                 : 0;
        if (h->p.autotune == 1) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            OuterRec rec;
            rec.mapping = h->outer_spmv_tpr;
            memcpy(rec.us, h->outer_us, sizeof rec.us);
            if (g_tune_outer.size() < 4096) g_tune_outer.emplace_back(okey, rec);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    return BAMG_OK;
}

// Fields on disjoint node sets: the graph of the diagonal field blocks of a
// level (the stored blocks between two nodes of one field), on which every
// field is aggregated and coloured separately (Sec. 4.3.1).  The graph is the
// disjoint union of the fields' graphs in contiguous node ranges, so the
// ascending-order rules of aggregation and colouring treat each field as if
// it were alone, and aggregate ids (ranks of the roots) run field by field.
static int level_field_graph(bamg_ctx* h, const Level& L, int** rp_f, int** ci_f, cudaStream_t s) {
    int *count = nullptr, *tmp = nullptr;
    const long sb = scan_tmp_bytes(L.n) + 64;
    TRY(h->alloc(rp_f, (size_t)L.n + 1));
    TRY(h->alloc(ci_f, (size_t)L.nnzb));
    TRY(h->alloc(&count, (size_t)L.n + 1));
    TRY(h->alloc(&tmp, (size_t)sb / sizeof(int) + 1));
    TRY(field_pattern(L.n, L.rp, L.ci, L.node_field, count, tmp, sb, *rp_f, *ci_f, s));
    h->release(count);
    h->release(tmp);
    return BAMG_OK;
}

// Start the first-fit colouring of level l (one field set) on its own stream
// from a second host thread; the result (the same colouring as on the setup
// stream) is taken by colour_join.  Without a thread the colouring runs on the
// setup stream at once.
static int colour_start(bamg_ctx* h, int l, Level& L, cudaStream_t s) {
    auto& j = h->cjob[l];
    TRY(h->alloc(&L.colour, (size_t)L.n));
    TRY(h->alloc(&j.flag, 4));
    TRY(h->alloc(&j.queue, 2 * (size_t)L.n));
    j.pin = reinterpret_cast<int*>(pin_slot());
    if (!j.pin) return BAMG_ECUDA;
    BAMG_CUDA_TRY(cudaStreamCreateWithFlags(&j.stream, cudaStreamNonBlocking));
    BAMG_CUDA_TRY(cudaEventCreateWithFlags(&j.ev, cudaEventDisableTiming));
    // the pattern and the stream-ordered allocations above come first
    BAMG_CUDA_TRY(cudaEventRecord(j.ev, s));
    BAMG_CUDA_TRY(cudaStreamWaitEvent(j.stream, j.ev, 0));
    int dev = 0;
    BAMG_CUDA_TRY(cudaGetDevice(&dev));
    const int n = L.n;
    const int *rp = L.rp, *ci = L.ci;
    int* colour = L.colour;
    auto* jp = &j;
    try {
        j.thread = std::thread([jp, dev, n, rp, ci, colour]() {
            int st = cudaSetDevice(dev) == cudaSuccess ? BAMG_OK : BAMG_ECUDA;
            if (st == BAMG_OK)
                st = colour_nodes(n, rp, ci, colour, jp->flag, jp->pin, jp->stream, &jp->n_colours, &jp->rounds,
                                  jp->queue);
            if (cudaEventRecord(jp->ev, jp->stream) != cudaSuccess && st == BAMG_OK) st = BAMG_ECUDA;
            jp->status = st;
        });
    } catch (...) {
        // no thread: colour on the setup stream now
        j.status = colour_nodes(n, rp, ci, colour, j.flag, j.pin, s, &j.n_colours, &j.rounds, j.queue);
        if (j.status == BAMG_OK) BAMG_CUDA_TRY(cudaEventRecord(j.ev, s));
    }
    return BAMG_OK;
}

// the colouring of level l started by colour_start, ordered before the setup
// stream's next work; *done false when none was started
static int colour_join(bamg_ctx* h, int l, Level& L, cudaStream_t s, bool* done) {
    auto& j = h->cjob[l];
    *done = false;
    if (!j.ev) return BAMG_OK;
    if (j.thread.joinable()) j.thread.join();
    TRY(j.status);
    BAMG_CUDA_TRY(cudaStreamWaitEvent(s, j.ev, 0));
    L.n_colours = j.n_colours;
    L.colour_rounds = j.rounds;
    h->release(j.flag);
    h->release(j.queue);
    j.flag = j.queue = nullptr;
    *done = true;
    return BAMG_OK;
}

// The tensor-core coarsest LU and inverse of a single system (FP32 coarsest
// solve of 224 to 2048 unknowns) enqueued on cap_stream, where it runs while
// the setup stream builds the finer levels' smoother data; the coarse branch
// of setup_impl joins it.  (The CUDA-core paths keep their place: their
// cooperative kernels want every CTA resident at once.)
static int coarse_begin(bamg_ctx* h, cudaStream_t s) {
    if (h->nsys > 1 || h->p.coarse_prec != 32 || h->p.coarse_tc != 1) return BAMG_OK;
    const Level& L = h->lev[h->nlev - 1];
    const long nd = (long)L.n * h->b;
    if (nd > kMaxCoarseDense || nd <= kCoarseTcMin || !tc_lu_supported((int)nd)) return BAMG_OK;
    h->nd = (int)nd;
    h->coarse_tc_used = true;
    TRY(h->alloc(&h->coarse_a, (size_t)(nd * nd)));
    TRY(h->alloc(&h->coarse_piv, (size_t)nd));
    TRY(h->alloc(&h->coarse_inv32, (size_t)(nd * nd)));
    TRY(h->alloc(&h->coarse_err, 4));
    float *a32 = nullptr, *lt32 = nullptr, *work32 = nullptr;
    TRY(h->alloc(&a32, (size_t)(nd * nd)));
    TRY(h->alloc(&lt32, (size_t)(nd * nd)));
    TRY(h->alloc(&work32, (size_t)tc_lu_scratch_floats((int)nd)));
    h->coarse_tmp = {a32, lt32, work32};
    BAMG_CUDA_TRY(cudaMemsetAsync(h->coarse_err, 0, 4 * sizeof(int), s));
    BAMG_CUDA_TRY(cudaEventCreateWithFlags(&h->coarse_ev, cudaEventDisableTiming));
    BAMG_CUDA_TRY(cudaEventRecord(h->coarse_ev, s));  // the coarsest values and the allocations above
    cudaStream_t cs = h->cap_stream;
    BAMG_CUDA_TRY(cudaStreamWaitEvent(cs, h->coarse_ev, 0));
    h->coarse_pending = true;
    TRY(coarse_dense(h->b, L.n, L.rp, L.ci, L.vals64, h->coarse_a, cs));
    TRY(launch_convert_d2f(nd * nd, h->coarse_a, a32, cs));
    TRY(dense_lu_inverse_tc((int)nd, a32, h->coarse_piv, h->coarse_inv32, lt32, work32, h->coarse_err, cs));
    BAMG_CUDA_TRY(cudaEventRecord(h->coarse_ev, cs));
    return BAMG_OK;
}

// the level-0 values on the device before their first use in the setup
static int vals_ready(bamg_ctx* h, cudaStream_t s) {
    if (!h->vals_pending) return BAMG_OK;
    h->vals_pending = false;
    BAMG_CUDA_TRY(cudaStreamWaitEvent(s, h->vals_ev, 0));
    return BAMG_OK;
}

static int setup_impl(bamg_ctx* h, const int* row_ptr, const int* col_idx, const double* vals, int n,
                      int nnzb, cudaStream_t s) {
    auto tp = Clock::now();
    const int b = h->b;
    const size_t bb = (size_t)b * b;
    TRY(h->alloc(&h->d_err, 4));
    h->h_pin = reinterpret_cast<int*>(pin_slot());
    h->h_scal = reinterpret_cast<double*>(pin_slot());
    if (!h->h_pin || !h->h_scal) return BAMG_ECUDA;
    BAMG_CUDA_TRY(cudaMemsetAsync(h->d_err, 0, 4 * sizeof(int), s));
    Level& L0 = h->lev[0];
    L0.n = n;
    L0.nnzb = nnzb;
    TRY(h->alloc(&L0.rp, (size_t)n + 1));
    TRY(h->alloc(&L0.ci, (size_t)nnzb));
    TRY(h->alloc(&L0.vals64, (size_t)nnzb * bb));
    BAMG_CUDA_TRY(cudaMemcpyAsync(L0.rp, row_ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, s));
    BAMG_CUDA_TRY(cudaMemcpyAsync(L0.ci, col_idx, sizeof(int) * (size_t)nnzb, cudaMemcpyDeviceToDevice, s));
    if (h->vals_host) {
        // host values: copied on the side stream after the stream-ordered
        // allocation above, overlapping the pattern phases below
        BAMG_CUDA_TRY(cudaEventCreateWithFlags(&h->vals_ev, cudaEventDisableTiming));
        BAMG_CUDA_TRY(cudaEventRecord(h->vals_ev, s));
        BAMG_CUDA_TRY(cudaStreamWaitEvent(h->cap_stream, h->vals_ev, 0));
        BAMG_CUDA_TRY(cudaMemcpyAsync(L0.vals64, h->vals_host, sizeof(double) * bb * nnzb, cudaMemcpyHostToDevice,
                                      h->cap_stream));
        BAMG_CUDA_TRY(cudaEventRecord(h->vals_ev, h->cap_stream));
        h->vals_pending = true;
    } else {
        BAMG_CUDA_TRY(cudaMemcpyAsync(L0.vals64, vals, sizeof(double) * bb * nnzb, cudaMemcpyDeviceToDevice, s));
    }
    // row_ptr consistency is checked on the host side of the device copy
    BAMG_CUDA_TRY(cudaMemcpyAsync(h->h_pin, L0.rp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA_TRY(cudaMemcpyAsync(h->h_pin + 1, L0.rp, sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (h->h_pin[0] != nnzb || h->h_pin[1] != 0) return BAMG_EINVAL;

    // node ranges of the systems on level 0 (one range for a single system)
    TRY(h->alloc(&L0.sys_off_d, L0.sys_off.size()));
    BAMG_CUDA_TRY(cudaMemcpyAsync(L0.sys_off_d, L0.sys_off.data(), sizeof(int) * L0.sys_off.size(),
                                  cudaMemcpyHostToDevice, s));
    if (h->nsys > 1) {  // every stored block stays inside its system
        int* node_sys = nullptr;
        TRY(h->alloc(&node_sys, (size_t)n));
        TRY(launch_fill_sys(h->nsys, L0.sys_off_d, 1, node_sys, s));
        TRY(launch_check_batch(n, L0.rp, L0.ci, node_sys, L0.sys_off_d, h->d_err, s));
        TRY(check_dev(h, s));
        h->release(node_sys);
    }

    if (h->nf > 1) {  // node ranges of the fields on level 0
        TRY(h->alloc(&L0.fo_d, L0.fo.size()));
        BAMG_CUDA_TRY(cudaMemcpyAsync(L0.fo_d, L0.fo.data(), sizeof(int) * L0.fo.size(), cudaMemcpyHostToDevice, s));
    }
    if (h->p.mlp) {  // FP16 copy of the network parameters
        float* p32 = nullptr;
        TRY(h->alloc(&p32, BAMG_MLP_NPARAMS));
        TRY(h->alloc(&h->mlp16, BAMG_MLP_NPARAMS));
        BAMG_CUDA_TRY(cudaMemcpyAsync(p32, h->p.mlp, sizeof(float) * BAMG_MLP_NPARAMS, cudaMemcpyHostToDevice, s));
        TRY(launch_pack_half(p32, h->mlp16, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        h->release(p32);
    }
    long long used_s = 0, used_p = 0;
    h->nlev = 1;
    for (int l = 0;; ++l) {
        Level& L = h->lev[l];
        TRY(h->alloc(&L.diag, (size_t)L.n));
        TRY(launch_check_pattern(L.n, L.rp, L.ci, L.diag, h->d_err, s));
        TRY(check_dev(h, s));
        h->t_phase[0] += ms_since(tp);
        tp = Clock::now();
        if (h->nf > 1) {
            TRY(h->alloc(&L.node_field, (size_t)L.n));
            TRY(launch_fill_sys(h->nf, L.fo_d, 1, L.node_field, s));
        }
        const bool coarsen = h->nlev < h->p.max_levels && (long)L.n * b > h->p.max_coarse && l + 1 < kMaxLevels;
        if (!coarsen) break;
        // aggregation (clone for every field: one aggregate map per level)
        AggWork w{};
        int *d_count = nullptr, *scan_tmp = nullptr;
        const long stb = scan_tmp_bytes(L.n) + 64;
        TRY(h->alloc(&w.state, (size_t)L.n));
        TRY(h->alloc(&w.rootid, (size_t)L.n + 1));
        TRY(h->alloc(&w.agg1, (size_t)L.n));
        TRY(h->alloc(&w.settled, (size_t)L.n));
        TRY(h->alloc(&w.flag, 4));
        TRY(h->alloc(&d_count, 4));
        TRY(h->alloc(&scan_tmp, (size_t)stb / sizeof(int) + 1));
        TRY(h->alloc(&L.agg, (size_t)L.n));
        w.host_flag = h->h_pin;
        BAMG_CUDA_TRY(cudaMemsetAsync(d_count, 0, 4 * sizeof(int), s));
        int rounds = 0;
        int *g_rp = L.rp, *g_ci = L.ci;
        if (h->nf > 1) TRY(level_field_graph(h, L, &g_rp, &g_ci, s));
        const int nc = aggregate_nodes(L.n, g_rp, g_ci, L.agg, w, d_count, scan_tmp, stb, s, &rounds);
        if (nc < 0) return nc;
        L.agg_rounds = rounds;
        if (h->nf > 1) {
            h->release(g_rp);
            h->release(g_ci);
            // node ranges of the fields on the coarse level: the aggregates of
            // a field are numbered by the ranks of its roots, a contiguous range
            Level& Cf = h->lev[l + 1];
            TRY(h->alloc(&Cf.fo_d, (size_t)h->nf + 1));
            TRY(launch_coarse_offsets(h->nf, L.fo_d, w.rootid, Cf.fo_d, s));
            Cf.fo.assign((size_t)h->nf + 1, 0);
            BAMG_CUDA_TRY(cudaMemcpyAsync(Cf.fo.data(), Cf.fo_d, sizeof(int) * (h->nf + 1), cudaMemcpyDeviceToHost, s));
            BAMG_CUDA_TRY(cudaStreamSynchronize(s));
            for (int g = 0; g < h->nf; ++g)
                if (Cf.fo[g + 1] <= Cf.fo[g]) return BAMG_ECUDA;  // every field keeps at least one node
            if (Cf.fo[0] != 0 || Cf.fo[h->nf] != nc) return BAMG_ECUDA;
        }
        // node ranges of the systems on the coarse level: the aggregates of a
        // system are numbered by the ranks of its roots, a contiguous range
        Level& Cn = h->lev[l + 1];
        TRY(h->alloc(&Cn.sys_off_d, (size_t)h->nsys + 1));
        TRY(launch_coarse_offsets(h->nsys, L.sys_off_d, w.rootid, Cn.sys_off_d, s));
        Cn.sys_off.assign((size_t)h->nsys + 1, 0);
        BAMG_CUDA_TRY(cudaMemcpyAsync(Cn.sys_off.data(), Cn.sys_off_d, sizeof(int) * (h->nsys + 1),
                                      cudaMemcpyDeviceToHost, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        h->release(w.state);
        h->release(w.rootid);
        h->release(w.agg1);
        h->release(w.settled);
        if (nc == 0 || nc == L.n) break;  // no coarsening possible
        L.n_agg = nc;
        TRY(h->alloc(&L.agg_ptr, (size_t)nc + 1));
        TRY(h->alloc(&L.members, (size_t)L.n));
        int* tmp = nullptr;
        TRY(h->alloc(&tmp, (size_t)nc + 1 + scan_tmp_bytes(nc) / sizeof(int) + 16));
        TRY(build_members(L.n, nc, L.agg, L.agg_ptr, L.members, tmp, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        h->t_phase[1] += ms_since(tp);
        tp = Clock::now();
        if (h->p.mlp) TRY(vals_ready(h, s));  // the features read the values
        TRY(level_weights(h, l, s, &used_s, &used_p));
        h->t_phase[7] += ms_since(tp);
        tp = Clock::now();
        if (L.smoothed) {
            TRY(vals_ready(h, s));
            TRY(smoothed_galerkin(h, l, s));
            h->release(w.flag);
            h->release(d_count);
            h->release(scan_tmp);
            h->release(tmp);
            h->nlev++;
            h->t_phase[2] += ms_since(tp);
            tp = Clock::now();
            continue;
        }
        // Galerkin product
        Level& C = h->lev[l + 1];
        C.n = nc;
        int *count = nullptr, *tmp_cols = nullptr;
        TRY(h->alloc(&count, (size_t)nc + 1));
        TRY(h->alloc(&tmp_cols, (size_t)nc * kRapCap));
        TRY(h->alloc(&C.rp, (size_t)nc + 1));
        TRY(rap_symbolic(nc, L.agg_ptr, L.members, L.rp, L.ci, L.agg, count, tmp_cols, kRapCap, h->d_err, s));
        TRY(check_dev(h, s));
        int* scan2 = nullptr;
        TRY(h->alloc(&scan2, (size_t)scan_tmp_bytes(nc) / sizeof(int) + 16));
        TRY(exclusive_scan(nc, count, C.rp, scan2, scan_tmp_bytes(nc) + 64, s));
        BAMG_CUDA_TRY(cudaMemcpyAsync(h->h_pin, C.rp + nc, sizeof(int), cudaMemcpyDeviceToHost, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        C.nnzb = h->h_pin[0];
        TRY(h->alloc(&C.ci, (size_t)C.nnzb));
        TRY(h->alloc(&C.vals64, (size_t)C.nnzb * bb));
        TRY(rap_fill_cols(nc, C.rp, tmp_cols, kRapCap, C.ci, s));
        TRY(vals_ready(h, s));  // the pattern phases above overlapped the copy of host values
        TRY(rap_numeric(b, nc, L.agg_ptr, L.members, L.rp, L.ci, L.vals64, L.agg, C.rp, C.ci, C.vals64, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        h->release(w.flag);
        h->release(d_count);
        h->release(scan_tmp);
        h->release(tmp);
        h->release(count);
        h->release(tmp_cols);
        h->release(scan2);
        h->nlev++;
        h->t_phase[2] += ms_since(tp);
        tp = Clock::now();
    }
    TRY(vals_ready(h, s));  // (a level that was not coarsened)
    for (int l = h->nlev - 1; l < kMaxLevels; ++l)  // a level that could not be coarsened keeps no smoother
        if (h->cjob[l].thread.joinable()) h->cjob[l].thread.join();
    if (!h->p.mlp && ((h->p.omega_s_arr && used_s != h->p.omega_s_len) ||
                      (h->p.smooth_p && h->p.omega_p_arr && used_p != h->p.omega_p_len)))
        return BAMG_EINVAL;  // the per-level arrays must match the hierarchy exactly
    // the caller's host arrays are not kept
    h->p.omega_s_arr = nullptr;
    h->p.omega_p_arr = nullptr;
    // every smoother level's colouring beside the coarsest LU and the smoother
    // data (the aggregation and Galerkin products above ran alone)
    if (h->nf == 1)
        for (int l = 0; l + 1 < h->nlev; ++l) TRY(colour_start(h, l, h->lev[l], s));
    TRY(coarse_begin(h, s));
    h->p.mlp = nullptr;
    // smoother data on every level but the coarsest
    for (int l = 0; l + 1 < h->nlev; ++l) {
        Level& L = h->lev[l];
        bool coloured = false;
        TRY(colour_join(h, l, L, s, &coloured));
        if (!coloured) {
            TRY(h->alloc(&L.colour, (size_t)L.n));
            int *cflag = nullptr, *queue = nullptr;
            TRY(h->alloc(&cflag, 4));
            TRY(h->alloc(&queue, 2 * (size_t)L.n));
            int rounds = 0;
            int *g_rp = L.rp, *g_ci = L.ci;
            if (h->nf > 1) TRY(level_field_graph(h, L, &g_rp, &g_ci, s));
            TRY(colour_nodes(L.n, g_rp, g_ci, L.colour, cflag, h->h_pin, s, &L.n_colours, &rounds, queue));
            L.colour_rounds = rounds;
            h->release(cflag);
            h->release(queue);
            if (h->nf > 1) {
                h->release(g_rp);
                h->release(g_ci);
            }
        }
        if (h->nf > 1) {
            // first-fit colours per field, shifted so that field g's colours
            // follow those of fields 0..g-1
            int* cm = nullptr;
            TRY(h->alloc(&cm, (size_t)h->nf + 1));
            TRY(field_colour_counts(L.n, h->nf, L.colour, L.node_field, cm, s));
            std::vector<int> cnt((size_t)h->nf, 0);
            BAMG_CUDA_TRY(cudaMemcpyAsync(cnt.data(), cm, sizeof(int) * h->nf, cudaMemcpyDeviceToHost, s));
            BAMG_CUDA_TRY(cudaStreamSynchronize(s));
            L.fcol.assign((size_t)h->nf + 1, 0);
            for (int g = 0; g < h->nf; ++g) {
                if (cnt[g] < 1) return BAMG_ECUDA;
                L.fcol[g + 1] = L.fcol[g] + cnt[g];
            }
            BAMG_CUDA_TRY(cudaMemcpyAsync(cm, L.fcol.data(), sizeof(int) * h->nf, cudaMemcpyHostToDevice, s));
            TRY(field_colour_shift(L.n, cm, L.node_field, L.colour, s));
            BAMG_CUDA_TRY(cudaStreamSynchronize(s));
            h->release(cm);
            L.n_colours = L.fcol[h->nf];
        }
        TRY(h->alloc(&L.colour_ptr_d, (size_t)L.n_colours + 1));
        TRY(h->alloc(&L.colour_nodes, (size_t)L.n));
        int* tmp = nullptr;
        TRY(h->alloc(&tmp, (size_t)L.n + 1 + scan_tmp_bytes(L.n) / sizeof(int) + 16));
        TRY(colour_order(L.n, L.n_colours, L.colour, L.colour_ptr_d, L.colour_nodes, tmp, s));
        L.colour_ptr.assign(L.n_colours + 1, 0);
        BAMG_CUDA_TRY(cudaMemcpyAsync(L.colour_ptr.data(), L.colour_ptr_d, sizeof(int) * (L.n_colours + 1),
                                      cudaMemcpyDeviceToHost, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        h->release(tmp);
        if (L.colour_ptr[L.n_colours] != L.n) return BAMG_ECUDA;
        TRY(h->alloc(&L.lowk, (size_t)L.nnzb));
        if (h->nf > 1) TRY(field_lower_flags(L.n, L.rp, L.ci, L.colour, L.node_field, L.lowk, s));
        else TRY(launch_lower_flags(L.n, L.rp, L.ci, L.colour, L.lowk, s));
        TRY(build_sweep_plan(h, L, s));
        {
            int* mr = nullptr;
            TRY(h->alloc(&mr, 1));
            TRY(launch_row_len_max(L.n, L.rp, mr, s));
            BAMG_CUDA_TRY(cudaMemcpyAsync(h->h_pin, mr, sizeof(int), cudaMemcpyDeviceToHost, s));
            BAMG_CUDA_TRY(cudaStreamSynchronize(s));
            L.max_row = h->h_pin[0];
            h->release(mr);
        }
        h->t_phase[3] += ms_since(tp);
        tp = Clock::now();
        if (!L.dinv64) {  // (already there when P was smoothed)
            TRY(h->alloc(&L.dinv64, (size_t)L.n * h->F * h->fb * h->fb));
            TRY(block_inverses(b, h->fb, L.n, L.diag, L.vals64, L.dinv64, h->d_err, s));
            TRY(check_dev(h, s));
        }
        if (h->p.sub_solver == 1) {  // ILU(0) of every field's A_ff in colour order
            const size_t nlu = (size_t)h->F * L.nnzb * h->fb * h->fb;
            TRY(h->alloc(&L.pos, (size_t)L.n));
            TRY(h->alloc(&L.ilu64, nlu));
            TRY(h->alloc(&L.upk, (size_t)L.nnzb));
            const int* nfield = h->nf > 1 ? L.node_field : nullptr;
            TRY(ilu_factor(L.n, b, h->fb, h->F, L.nnzb, L.n_colours, L.colour_ptr, L.colour_nodes, L.rp, L.ci,
                           L.diag, nfield, L.vals64, L.pos, L.ilu64, h->d_err, s));
            TRY(launch_upper_flags(L.n, L.rp, L.ci, L.colour, nfield, L.upk, s));
            TRY(check_dev(h, s));
            if (h->p.cycle_prec == 32) {
                TRY(h->alloc(&L.ilu32, nlu));
                TRY(launch_convert_d2f((long)nlu, L.ilu64, L.ilu32, s));
            }
        }
        if (h->p.sub_solver == 2) TRY(schwarz_level(h, l, s));
        if (h->p.cycle_prec == 32 && L.omega_s64) {
            TRY(h->alloc(&L.omega_s32, (size_t)L.n * h->F));
            TRY(launch_convert_d2f((long)L.n * h->F, L.omega_s64, L.omega_s32, s));
        }
        if (h->p.cycle_prec == 32) {
            TRY(h->alloc(&L.vals32, (size_t)L.nnzb * bb));
            TRY(h->alloc(&L.dinv32, (size_t)L.n * h->F * h->fb * h->fb));
            // field-major rows on levels larger than L2 (a field step streams
            // contiguous runs there; see vrow)
            int l2 = 0, dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
                l2 = 0;
            L.fm = h->F > 1 && (h->p.value_layout == 2 ||
                                (h->p.value_layout == 0 && l2 > 0 && (double)L.nnzb * bb * sizeof(float) > (double)l2));
            if (L.fm)
                TRY(launch_convert_fieldmajor(L.n, b, h->fb, L.rp, L.vals64, L.vals32, s));
            else
                TRY(launch_convert_d2f((long)L.nnzb * bb, L.vals64, L.vals32, s));
            TRY(launch_convert_d2f((long)L.n * h->F * h->fb * h->fb, L.dinv64, L.dinv32, s));
        }
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        h->t_phase[4] += ms_since(tp);
        tp = Clock::now();
    }
    // coarsest level of a batch: one dense FP64 LU and inverse per system
    if (h->nsys > 1) {
        Level& L = h->lev[h->nlev - 1];
        std::vector<long> inv_off((size_t)h->nsys + 1, 0);
        int max_nd = 0;
        for (int q = 0; q < h->nsys; ++q) {
            const long nd = (long)(L.sys_off[q + 1] - L.sys_off[q]) * b;
            if (nd > kMaxCoarseDense) return BAMG_EUNSUPPORTED;
            max_nd = nd > max_nd ? (int)nd : max_nd;
            inv_off[q + 1] = inv_off[q] + nd * nd;
        }
        h->nd_total = L.n * b;
        TRY(h->alloc(&h->inv_off_d, inv_off.size()));
        BAMG_CUDA_TRY(cudaMemcpyAsync(h->inv_off_d, inv_off.data(), sizeof(long) * inv_off.size(),
                                      cudaMemcpyHostToDevice, s));
        TRY(h->alloc(&h->binv, (size_t)inv_off.back()));
        TRY(h->alloc(&h->row_sys_d, (size_t)h->nd_total));
        TRY(launch_fill_sys(h->nsys, L.sys_off_d, b, h->row_sys_d, s));
        double *work = nullptr, *col = nullptr;
        int* piv = nullptr;
        TRY(h->alloc(&work, max_nd > 156 ? (size_t)inv_off.back() : 1));
        TRY(h->alloc(&col, (size_t)h->nd_total));
        TRY(h->alloc(&piv, (size_t)h->nd_total));
        TRY(batched_lu_inverse(h->nsys, b, max_nd, L.sys_off_d, h->inv_off_d, L.rp, L.ci, L.vals64, work, h->binv,
                               piv, col, h->d_err, s));
        TRY(check_dev(h, s));
        h->release(work);
        h->release(col);
        h->release(piv);
        h->nd = 0;
        h->t_phase[5] += ms_since(tp);
        tp = Clock::now();
    } else if (h->coarse_pending) {
        // the tensor-core LU enqueued by coarse_begin
        BAMG_CUDA_TRY(cudaStreamWaitEvent(s, h->coarse_ev, 0));
        h->coarse_pending = false;
        BAMG_CUDA_TRY(cudaMemcpyAsync(h->h_pin, h->coarse_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        TRY(map_dev_error(h->h_pin[0]));
        for (void* q : h->coarse_tmp) h->release(q);
        h->coarse_tmp.clear();
        h->t_phase[5] += ms_since(tp);
        tp = Clock::now();
    } else {
        Level& L = h->lev[h->nlev - 1];
        const long nd = (long)L.n * b;
        if (nd > kMaxCoarseDense) return BAMG_EUNSUPPORTED;
        h->nd = (int)nd;
        TRY(h->alloc(&h->coarse_a, (size_t)(nd * nd)));
        TRY(h->alloc(&h->coarse_piv, (size_t)nd));
        double* col = nullptr;
        TRY(h->alloc(&col, (size_t)dense_lu_scratch((int)nd)));
        TRY(coarse_dense(b, L.n, L.rp, L.ci, L.vals64, h->coarse_a, s));
        if (h->p.coarse_prec == 32) {
            float *a32 = nullptr, *lt32 = nullptr;
            TRY(h->alloc(&a32, (size_t)(nd * nd)));
            TRY(h->alloc(&lt32, (size_t)(nd * nd)));
            TRY(h->alloc(&h->coarse_inv32, (size_t)(nd * nd)));
            TRY(launch_convert_d2f(nd * nd, h->coarse_a, a32, s));
            h->coarse_tc_used = h->p.coarse_tc == 1 && nd > kCoarseTcMin && tc_lu_supported((int)nd);
            if (h->coarse_tc_used) {
                float* work32 = nullptr;
                TRY(h->alloc(&work32, (size_t)tc_lu_scratch_floats((int)nd)));
                TRY(dense_lu_inverse_tc((int)nd, a32, h->coarse_piv, h->coarse_inv32, lt32, work32, h->d_err, s));
                TRY(check_dev(h, s));
                h->release(work32);
            } else {
                TRY(dense_lu_inverse<float>((int)nd, a32, h->coarse_piv, h->coarse_inv32, lt32, col, h->d_err, s));
                TRY(check_dev(h, s));
            }
            h->release(lt32);
            h->release(a32);
        } else {
            double* lt = nullptr;
            TRY(h->alloc(&h->coarse_inv, (size_t)(nd * nd)));
            TRY(h->alloc(&lt, (size_t)(nd * nd)));
            TRY(dense_lu_inverse<double>((int)nd, h->coarse_a, h->coarse_piv, h->coarse_inv, lt, col, h->d_err, s));
            TRY(check_dev(h, s));
            h->release(lt);
        }
        h->release(col);
        h->t_phase[5] += ms_since(tp);
        tp = Clock::now();
    }
    // work vectors in the cycle precision
    const size_t es = h->p.cycle_prec == 32 ? sizeof(float) : sizeof(double);
    for (int l = 0; l < h->nlev; ++l) {
        Level& L = h->lev[l];
        const size_t nb = (size_t)L.n * b;
        char* q = nullptr;
        if (l + 1 < h->nlev) {
            TRY(h->alloc(&q, nb * es)); L.xa = q;
            TRY(h->alloc(&q, nb * es)); L.xb = q;
            TRY(h->alloc(&q, (size_t)L.n * h->fb * es)); L.xt = q;
            TRY(h->alloc(&q, nb * es)); L.res = q;
        }
        if (l > 0) {
            TRY(h->alloc(&q, nb * es)); L.rhs = q;
            TRY(h->alloc(&q, nb * es)); L.uc = q;
        }
    }
    const size_t N = (size_t)n * b;
    TRY(h->alloc(&h->cyc_in, N));
    TRY(h->alloc(&h->cyc_out, N));
    if (h->p.cycle_prec == 32) {
        TRY(h->alloc(&h->r32, N));
        TRY(h->alloc(&h->z32, N));
    }
    // chunks of the level-0 vectors for the per-system reductions
    {
        std::vector<int> csys, sc(1, 0);
        std::vector<long> ce0, ce1;
        const long kChunk = 4096;
        for (int q = 0; q < h->nsys; ++q) {
            const long e0 = (long)L0.sys_off[q] * b, e1 = (long)L0.sys_off[q + 1] * b;
            for (long e = e0; e < e1; e += kChunk) {
                csys.push_back(q);
                ce0.push_back(e);
                ce1.push_back(e + kChunk < e1 ? e + kChunk : e1);
            }
            sc.push_back((int)csys.size());
        }
        int *d_csys = nullptr, *d_sc = nullptr;
        long *d_e0 = nullptr, *d_e1 = nullptr;
        TRY(h->alloc(&d_csys, csys.size()));
        TRY(h->alloc(&d_sc, sc.size()));
        TRY(h->alloc(&d_e0, ce0.size()));
        TRY(h->alloc(&d_e1, ce1.size()));
        BAMG_CUDA_TRY(cudaMemcpyAsync(d_csys, csys.data(), sizeof(int) * csys.size(), cudaMemcpyHostToDevice, s));
        BAMG_CUDA_TRY(cudaMemcpyAsync(d_sc, sc.data(), sizeof(int) * sc.size(), cudaMemcpyHostToDevice, s));
        BAMG_CUDA_TRY(cudaMemcpyAsync(d_e0, ce0.data(), sizeof(long) * ce0.size(), cudaMemcpyHostToDevice, s));
        BAMG_CUDA_TRY(cudaMemcpyAsync(d_e1, ce1.data(), sizeof(long) * ce1.size(), cudaMemcpyHostToDevice, s));
        h->seg = SegTable{h->nsys, (int)csys.size(), d_csys, d_e0, d_e1, d_sc};
    }
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (h->p.autotune >= 1) {
        if (h->p.cycle_prec == 64) TRY(autotune_levels<double>(h, s));
        else TRY(autotune_levels<float>(h, s));
    }
    if (h->nsys == 1 && h->nf == 1) TRY(setup_tail(h, s));
    h->t_phase[6] += ms_since(tp);
    return BAMG_OK;
}

// vals_on_host: vals is a host array (the host-buffer entry points); its copy
// to the device overlaps the setup's pattern phases
static int setup_common(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int nnzb, int b,
                        const int* field_of_dof, const amg_params* p, void* stream, bamg_t* out, int nsys,
                        const int* sys_node_off, int nf = 1, const int* field_node_off = nullptr,
                        bool vals_on_host = false) {
    if (!out) return BAMG_EINVAL;
    *out = nullptr;
    if (!row_ptr || !col_idx || !vals || !field_of_dof || n_nodes < 1 || nnzb < n_nodes || b < 1 || b > kMaxB)
        return BAMG_EINVAL;
    if (nsys < 1 || nsys > n_nodes) return BAMG_EINVAL;
    if (nsys > 1) {
        if (!sys_node_off || sys_node_off[0] != 0 || sys_node_off[nsys] != n_nodes) return BAMG_EINVAL;
        for (int q = 0; q < nsys; ++q)
            if (sys_node_off[q + 1] <= sys_node_off[q]) return BAMG_EINVAL;
    }
    amg_params prm;
    if (p) prm = *p;
    else amg_default_params(&prm);
    if (prm.max_levels < 1 || prm.max_levels > kMaxLevels || prm.n_pre < 0 || prm.n_post < 0 ||
        !(prm.omega > 0.0) || (prm.cycle_prec != 32 && prm.cycle_prec != 64) || prm.tail_dofs < 0 ||
        prm.autotune < 0 || prm.autotune > 8 || (prm.smooth_p != 0 && prm.smooth_p != 1) ||
        !std::isfinite(prm.omega_p) || (prm.pr_storage != 32 && prm.pr_storage != 16) ||
        (prm.pr_storage == 16 && prm.cycle_prec != 32) || prm.omega_s_len < 0 || prm.omega_p_len < 0 ||
        (prm.omega_s_arr && prm.omega_s_len == 0) || (prm.omega_p_arr && !prm.smooth_p && !prm.mlp) ||
        prm.mlp_levels < 0 || (prm.use_pdl != 0 && prm.use_pdl != 1) ||
        (prm.coarse_prec != 64 && prm.coarse_prec != 32) || (prm.coarse_prec == 32 && prm.cycle_prec != 32) ||
        (prm.tail_grid != 0 && prm.tail_grid != 1) || prm.value_layout < 0 || prm.value_layout > 2 ||
        prm.sweep < 0 || prm.sweep > 3 || prm.sub_solver < 0 || prm.sub_solver > 2 ||
        prm.schwarz_overlap < 0 || prm.schwarz_overlap > 1 || prm.ortho < 0 || prm.ortho > 1 ||
        prm.coarse_tc < 0 || prm.coarse_tc > 1 || prm.inner_sweeps < 0 || prm.inner_sweeps > 64 ||
        (prm.inner_sweeps > 1 && (prm.sub_solver != 0 || nf > 1)))
        return BAMG_EINVAL;
    if (prm.inner_sweeps == 0) prm.inner_sweeps = 1;
    if (prm.sub_solver != 0 || prm.inner_sweeps > 1) {
        // the cycle with another sub-solve runs as separate launches: no
        // recorded single-launch tail, no persistent sweep
        prm.tail_dofs = 0;
        prm.tail_grid = 0;
        prm.sweep = 1;
    }
    // fields: non-decreasing 0..F-1 in unit steps, equal sizes
    if (field_of_dof[0] != 0) return BAMG_EINVAL;
    int F = 1;
    for (int d = 1; d < b; ++d) {
        const int step = field_of_dof[d] - field_of_dof[d - 1];
        if (step != 0 && step != 1) return BAMG_EINVAL;
        F = field_of_dof[d] + 1;
    }
    int fsize[kMaxB] = {}, fmax = 0;
    for (int d = 0; d < b; ++d) fmax = std::max(fmax, ++fsize[field_of_dof[d]]);
    bool unequal = false;
    for (int f = 0; f < F; ++f) unequal |= fsize[f] != fmax;
    if (unequal) {
        // fields of unequal size: set up the padded system with equal fields
        // (k_pad.cu); the options built on one common field size are refused
        if (nf > 1) return BAMG_EINVAL;
        if (prm.smooth_p || prm.mlp || prm.omega_p_arr || prm.sub_solver != 0) return BAMG_EUNSUPPORTED;
        const int bp = F * fmax;
        if (bp > kMaxB || !supported_block(bp, fmax)) return BAMG_EUNSUPPORTED;
        PadMap pm;
        pm.b = b;
        pm.bp = bp;
        int first[kMaxB];
        for (int f = F - 1; f >= 0; --f) first[f] = -1;
        for (int d = b - 1; d >= 0; --d) first[field_of_dof[d]] = d;
        for (int q = 0; q < bp; ++q) pm.src[q] = -1;
        for (int d = 0; d < b; ++d) {
            const int q = field_of_dof[d] * fmax + (d - first[field_of_dof[d]]);
            pm.dst[d] = (signed char)q;
            pm.src[q] = (signed char)d;
        }
        int fmap_p[kMaxB];
        for (int q = 0; q < bp; ++q) fmap_p[q] = q / fmax;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        double* vp = nullptr;
        double* vd = nullptr;  // host values: a device copy for the padding kernel
        if (pool_alloc((void**)&vp, sizeof(double) * (size_t)nnzb * bp * bp, s) != cudaSuccess) return BAMG_ECUDA;
        if (vals_on_host &&
            (pool_alloc((void**)&vd, sizeof(double) * (size_t)nnzb * b * b, s) != cudaSuccess ||
             cudaMemcpyAsync(vd, vals, sizeof(double) * (size_t)nnzb * b * b, cudaMemcpyHostToDevice, s) !=
                 cudaSuccess)) {
            if (vd) cudaFreeAsync(vd, s);
            cudaFreeAsync(vp, s);
            return BAMG_ECUDA;
        }
        int st = launch_pad_values(pm, n_nodes, nnzb, row_ptr, col_idx, vd ? vd : vals, vp, s);
        if (vd) cudaFreeAsync(vd, s);
        if (st == BAMG_OK)
            st = setup_common(row_ptr, col_idx, vp, n_nodes, nnzb, bp, fmap_p, &prm, stream, out, nsys, sys_node_off);
        cudaFreeAsync(vp, s);
        if (st != BAMG_OK) return st;
        bamg_ctx* h = *out;
        h->padded = true;
        h->pad = pm;
        const size_t NP = (size_t)n_nodes * bp;
        st = h->alloc(&h->pad_b, NP);
        if (st == BAMG_OK) st = h->alloc(&h->pad_x, NP);
        if (st != BAMG_OK) {
            amg_destroy(h);
            *out = nullptr;
        }
        return st;
    }
    const int fb = b / F;
    if (!supported_block(b, fb)) return BAMG_EUNSUPPORTED;
    // fields on disjoint node sets: contiguous non-empty node ranges, every dof
    // of a node in the node's field, one system, the plain method
    if (nf < 1 || nf > BAMG_MAX_NODE_FIELDS) return BAMG_EINVAL;
    if (nf > 1) {
        if (!field_node_off || field_node_off[0] != 0 || field_node_off[nf] != n_nodes || F != 1 || nsys != 1 ||
            prm.smooth_p || prm.mlp || prm.omega_s_arr || prm.omega_p_arr)
            return BAMG_EINVAL;
        for (int g = 0; g < nf; ++g)
            if (field_node_off[g + 1] <= field_node_off[g]) return BAMG_EINVAL;
        // the single-launch tail records no copies of the other fields' nodes
        prm.tail_dofs = 0;
        prm.tail_grid = 0;
    }
    bamg_ctx* h = new (std::nothrow) bamg_ctx();
    if (!h) return BAMG_ECUDA;
    h->b = b;
    h->F = F;
    h->fb = fb;
    h->p = prm;
    h->nsys = nsys;
    if (nsys > 1) h->lev[0].sys_off.assign(sys_node_off, sys_node_off + nsys + 1);
    else h->lev[0].sys_off = {0, n_nodes};
    h->nf = nf;
    if (nf > 1) h->lev[0].fo.assign(field_node_off, field_node_off + nf + 1);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->stream = s;
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return BAMG_ECUDA;
    }
    if (vals_on_host) h->vals_host = vals;
    int st = setup_impl(h, row_ptr, col_idx, vals, n_nodes, nnzb, s);
    h->vals_host = nullptr;  // not kept
    if (st != BAMG_OK) {
        cudaStreamSynchronize(s);
        delete h;
        return st;
    }
    *out = h;
    return BAMG_OK;
}

extern "C" int amg_setup(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int nnzb,
                         int b, const int* field_of_dof, const amg_params* p, void* stream, bamg_t* out) {
    return setup_common(row_ptr, col_idx, vals, n_nodes, nnzb, b, field_of_dof, p, stream, out, 1, nullptr);
}

extern "C" int amg_setup_batched(int nsys, const int* sys_node_off, const int* row_ptr, const int* col_idx,
                                 const double* vals, int n_nodes, int nnzb, int b, const int* field_of_dof,
                                 const amg_params* p, void* stream, bamg_t* out) {
    return setup_common(row_ptr, col_idx, vals, n_nodes, nnzb, b, field_of_dof, p, stream, out, nsys, sys_node_off);
}

static int setup_fields(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int nnzb, int b,
                        int n_fields, const int* field_node_off, const amg_params* p, void* stream, bamg_t* out,
                        bool vals_on_host) {
    if (!out) return BAMG_EINVAL;
    *out = nullptr;
    if (b < 1 || b > kMaxB || n_fields < 1 || !field_node_off) return BAMG_EINVAL;
    int zeros[kMaxB] = {};
    return setup_common(row_ptr, col_idx, vals, n_nodes, nnzb, b, zeros, p, stream, out, 1, nullptr, n_fields,
                        field_node_off, vals_on_host);
}

extern "C" int amg_setup_fields(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int nnzb,
                                int b, int n_fields, const int* field_node_off, const amg_params* p, void* stream,
                                bamg_t* out) {
    return setup_fields(row_ptr, col_idx, vals, n_nodes, nnzb, b, n_fields, field_node_off, p, stream, out, false);
}

extern "C" int amg_level_fields(bamg_t h, int level, int* node_off, int* colour_off) {
    if (!h || level < 0 || level >= h->nlev) return BAMG_EINVAL;
    const Level& L = h->lev[level];
    const bool smoother = level + 1 < h->nlev;
    for (int g = 0; g <= h->nf; ++g) {
        if (node_off) node_off[g] = h->nf > 1 ? L.fo[g] : (g == 0 ? 0 : L.n);
        if (colour_off) colour_off[g] = !smoother ? 0 : h->nf > 1 ? L.fcol[g] : (g == 0 ? 0 : L.n_colours);
    }
    return h->nf;
}

extern "C" int amg_destroy(bamg_t h) {
    if (!h) return BAMG_OK;
    cudaStreamSynchronize(h->stream);
    delete h;
    return BAMG_OK;
}

// ---------------------------------------------------------------------------
// V-cycle
// ---------------------------------------------------------------------------

// A V-cycle step is launched now or, while h->rec is set, appended to the
// phase list of the cluster tail kernel (with its algorithmic bytes / flops).
static void record(bamg_ctx* h, const TailPhase& ph, double bytes, double flops) {
    h->rec->push_back(ph);
    h->rec_bytes += bytes;
    h->rec_flops += flops;
}

// the field steps of one sweep of Algorithm 1: fields on node sets, else the
// dof fields of a node
static int field_steps(const bamg_ctx* h) { return h->nf > 1 ? h->nf : h->F; }

// Fields on node sets: a field step writes only the nodes of its own field.
// The other fields' nodes of x_out take x_in (plus the coarse correction P u_c
// in the first post-smoothing step), or zero from the zero initial guess.
template <typename T>
static int other_fields(bamg_ctx* h, const Level& L, int f, const T* x_in, T* x_out, const T* uc, cudaStream_t s) {
    const int b = h->b;
    for (int g = 0; g < h->nf; ++g) {
        if (g == f) continue;
        const int n_g = L.fo[g + 1] - L.fo[g];
        const size_t e0 = (size_t)L.fo[g] * b;
        // one kernel (copy, plus the coarse correction in the first
        // post-smoothing step): launched like the smoother's kernels, so the
        // cycle keeps its programmatic dependent launches
        TRY(launch_copy_prolong<T>(b, n_g, L.agg + L.fo[g], x_in ? x_in + e0 : nullptr, uc, x_out + e0, s));
    }
    return BAMG_OK;
}

// one field step of Algorithm 1 on level l: x_out = x_in updated in field f
// uc != nullptr: the coarse correction P uc is added to x_in on the fly (x_in is
// then the state before prolongation and x_out receives the corrected values)
// With fields on node sets, field f is the node range fo[f].. and its colours
// are fcol[f]..fcol[f+1]-1; each node is one b x b sub-solve block.
template <typename T>
static int bgs_step(bamg_ctx* h, int l, int f, const T* rhs, const T* x_in, T* x_out, const T* uc,
                    cudaStream_t s) {
    const Level& L = h->lev[l];
    const bool have_counts = (int)L.colour_nnz.size() == L.n_colours;
    const bool nodef = h->nf > 1;
    const int c_lo = nodef ? L.fcol[f] : 0, c_hi = nodef ? L.fcol[f + 1] : L.n_colours;
    if (h->p.sub_solver == 1) {
        // ILU(0) of A_ff: forward solve over the colours ascending (the field's
        // residual formed on the fly), backward solve descending, then x_f += omega x~
        const T* lu = level_ilu<T>(L) + (nodef ? 0 : (size_t)f * L.nnzb * h->fb * h->fb);
        for (int pass = 0; pass < 2; ++pass)
            for (int t = 0; t < c_hi - c_lo; ++t) {
                const int c = pass == 0 ? c_lo + t : c_hi - 1 - t;
                BgsArgs a;
                a.n_in_colour = L.colour_ptr[c + 1] - L.colour_ptr[c];
                a.nodes = L.colour_nodes + L.colour_ptr[c];
                a.colour = c;
                a.colours = L.colour;
                a.lowk = L.lowk;
                a.fm = level_fm<T>(L);
                a.rp = L.rp;
                a.ci = L.ci;
                a.vals = level_vals<T>(L);
                a.rhs = rhs;
                a.x_in = x_in;
                a.x_out = x_out;
                a.xt = L.xt;
                a.uc = uc;
                a.agg = uc ? L.agg : nullptr;
                a.field = nodef ? 0 : f;
                a.F = h->F;
                a.omega = h->p.omega;
                a.omega_node = level_omega<T>(L);
                double bytes = 0.0, flops = 0.0;
                if (h->prof && have_counts) {
                    const double es = sizeof(T), B = h->b, FB = h->fb, nc = a.n_in_colour;
                    const double nnz = (double)L.colour_nnz[c], low = (double)L.colour_nnz_lower[c];
                    const double up = nnz - low - nc;
                    if (pass == 0) {
                        bytes = nnz * 5.0 + (x_in ? nnz * FB * B * es + nnz * B * es : 0.0) + low * FB * FB * es +
                                low * FB * es + nc * (FB * FB * es + 12.0 + B * es + FB * es);
                        flops = 2.0 * ((x_in ? nnz * FB * B : 0.0) + low * FB * FB + nc * FB * FB / 2.0);
                    } else {
                        bytes = nnz * 5.0 + up * FB * FB * es + up * FB * es +
                                nc * (FB * FB * es + 12.0 + 2.0 * FB * es + (x_in ? 2.0 : 1.0) * B * es);
                        flops = 2.0 * (up * FB * FB + nc * FB * FB / 2.0);
                    }
                }
                PL(BAMG_K_SMOOTH, bytes, flops, launch_ilu_colour<T>(h->b, h->fb, a, lu, L.diag, L.upk, pass == 1, s));
            }
        if (nodef) TRY(other_fields<T>(h, L, f, x_in, x_out, uc, s));
        return BAMG_OK;
    }
    if (h->p.sub_solver == 2) {
        // restricted Schwarz: the field's residual, then every subdomain of the
        // field's aggregates at once; x_f += omega x~ for the own nodes
        const int fstep = nodef ? 0 : f;
        const int i0 = nodef ? L.fo[f] : 0, ni = nodef ? L.fo[f + 1] - L.fo[f] : L.n;
        T* rf = static_cast<T*>(L.xt);
        const double es = sizeof(T), B = h->b, FB = h->fb;
        PL(BAMG_K_SMOOTH,
           x_in ? (double)ni * (9.0 * (B * FB * es + 4.0 + B * es)) + ni * (8.0 + B * es + FB * es)
                : ni * (B * es + FB * es),
           x_in ? 2.0 * ni * 9.0 * B * FB : 0.0,
           launch_field_residual<T>(h->b, h->fb, level_fm<T>(L), ni, fstep, L.rp + i0, L.ci, level_vals<T>(L),
                                    x_in, uc, uc ? L.agg : nullptr, rhs + (size_t)i0 * h->b, rf + (size_t)i0 * h->fb,
                                    s));
        SchwarzArgs sa;
        if (nodef) {
            const Level& Cn = h->lev[l + 1];
            sa.agg_lo = Cn.fo[f];
            sa.agg_hi = Cn.fo[f + 1];
        } else {
            sa.agg_lo = 0;
            sa.agg_hi = L.n_agg;
        }
        sa.nfs = nodef ? 1 : h->F;
        sa.b = h->b;
        sa.fb = h->fb;
        sa.sd_ptr = L.sd_ptr;
        sa.sd_nodes = L.sd_nodes;
        sa.agg_ptr = L.agg_ptr;
        sa.members = L.members;
        sa.x_off = L.sd_xoff;
        sa.X = h->p.cycle_prec == 32 ? (const void*)L.sd_x32 : (const void*)L.sd_x64;
        sa.rf = rf;
        BgsArgs a;
        a.rhs = rhs;
        a.x_in = x_in;
        a.x_out = x_out;
        a.uc = uc;
        a.agg = uc ? L.agg : nullptr;
        a.field = fstep;
        a.F = h->F;
        a.omega = h->p.omega;
        a.omega_node = level_omega<T>(L);
        const double xb = (double)L.sd_xtotal / (nodef ? 1.0 : h->F) * es;
        PL(BAMG_K_SMOOTH, xb + (double)ni * (FB * es * 2.0 + B * es * (x_in ? 2.0 : 1.0)),
           2.0 * (double)L.sd_xtotal / (nodef ? 1.0 : h->F), launch_schwarz_apply<T>(sa, a, s));
        if (nodef) TRY(other_fields<T>(h, L, f, x_in, x_out, uc, s));
        return BAMG_OK;
    }
    if (h->p.inner_sweeps > 1) {
        // the sub-solve iterated: r_f = b_f - A_f* x_in for every node first (in
        // the level's residual buffer, unused while the level smooths), then
        // inner_sweeps multicolour sweeps on A_ff x~ = r_f, one launch per
        // colour; the last sweep writes x_out
        T* rf = static_cast<T*>(L.res);
        const double es = sizeof(T), B = h->b, FB = h->fb, nn = L.n, nz = L.nnzb;
        PL(BAMG_K_SMOOTH,
           nn * (8.0 + 2.0 * FB * es) + (x_in ? nz * (FB * B * es + 4.0 + B * es) : 0.0) +
               (x_in && uc ? nz * (4.0 + B * es) : 0.0),
           x_in ? 2.0 * nz * FB * B : 0.0,
           launch_field_residual<T>(h->b, h->fb, level_fm<T>(L), L.n, f, L.rp, L.ci, level_vals<T>(L), x_in, uc,
                                    uc ? L.agg : nullptr, rhs, rf, s));
        const int K = h->p.inner_sweeps;
        for (int q = 0; q < K; ++q)
            for (int c = 0; c < L.n_colours; ++c) {
                BgsArgs a;
                a.n_in_colour = L.colour_ptr[c + 1] - L.colour_ptr[c];
                a.nodes = L.colour_nodes + L.colour_ptr[c];
                a.colour = c;
                a.colours = L.colour;
                a.lowk = L.lowk;
                a.fm = level_fm<T>(L);
                a.rp = L.rp;
                a.ci = L.ci;
                a.vals = level_vals<T>(L);
                a.dinv = level_dinv<T>(L);
                a.rhs = rhs;
                a.x_in = x_in;
                a.x_out = x_out;
                a.xt = L.xt;
                a.uc = uc;
                a.agg = uc ? L.agg : nullptr;
                a.field = f;
                a.F = h->F;
                a.omega = h->p.omega;
                a.omega_node = level_omega<T>(L);
                double bytes = 0.0, flops = 0.0;
                if (h->prof && have_counts) {
                    const double nc = a.n_in_colour;
                    const double used = (q == 0 ? (double)L.colour_nnz_lower[c] : (double)L.colour_nnz[c] - nc);
                    bytes = (double)L.colour_nnz[c] * (q == 0 ? 1.0 : 4.0) + used * (4.0 + FB * FB * es + FB * es) +
                            nc * (12.0 + 3.0 * FB * es + FB * FB * es);
                    if (q == K - 1) bytes += nc * (B * es + (x_in ? B * es : 0.0) + (x_in && uc ? 4.0 + B * es : 0.0));
                    flops = 2.0 * (used + nc) * FB * FB;
                }
                PL(BAMG_K_SMOOTH, bytes, flops,
                   launch_gs_inner<T>(h->b, h->fb, a, rf, q == 0, q == K - 1, s));
            }
        return BAMG_OK;
    }
    if (L.sweep && L.sw_tiles > 0 && !h->rec) {
        // every colour of the step in one persistent launch
        BgsArgs a;
        a.nodes = L.colour_nodes;
        a.colours = L.colour;
        a.lowk = L.lowk;
        a.fm = level_fm<T>(L);
        a.rp = L.rp;
        a.ci = L.ci;
        a.vals = level_vals<T>(L);
        a.dinv = level_dinv<T>(L);
        a.rhs = rhs;
        a.x_in = x_in;
        a.x_out = x_out;
        a.xt = L.xt;
        a.uc = uc;
        a.agg = uc ? L.agg : nullptr;
        a.field = nodef ? 0 : f;
        a.F = h->F;
        a.omega = h->p.omega;
        a.omega_node = level_omega<T>(L);
        double bytes = 0.0, flops = 0.0;
        if (h->prof && have_counts)
            for (int c = c_lo; c < c_hi; ++c) {
                const double es = sizeof(T), B = h->b, FB = h->fb, nc = L.colour_ptr[c + 1] - L.colour_ptr[c];
                const double nnz = (double)L.colour_nnz[c], low = (double)L.colour_nnz_lower[c];
                bytes += nnz * (FB * B * es + 4.0) + nc * 8.0 + nc * FB * FB * es + nc * FB * es +
                         (x_in ? nc * B * es : 0.0) + nc * B * es + nc * FB * es + (c > 0 ? nc * FB * es : 0.0) +
                         (uc ? nc * (B * es + 4.0) : 0.0);
                flops += 2.0 * ((x_in ? nnz * FB * B : 0.0) + low * FB * FB + nc * FB * FB);
            }
        const SweepArgs sw = sweep_args(h, L, c_lo, c_hi);
        PL(BAMG_K_SMOOTH, bytes, flops,
           launch_bgs_sweep<T>(h->b, h->fb, a, sw, L.sw_tile_ptr[c_hi] - L.sw_tile_ptr[c_lo], L.sweep == 2, s));
        if (nodef) TRY(other_fields<T>(h, L, f, x_in, x_out, uc, s));
        return BAMG_OK;
    }
    for (int c = c_lo; c < c_hi; ++c) {
        BgsArgs a;
        a.n_in_colour = L.colour_ptr[c + 1] - L.colour_ptr[c];
        a.nodes = L.colour_nodes + L.colour_ptr[c];
        a.colour = c;
        a.colours = L.colour;
        a.lowk = L.lowk;
        a.fm = level_fm<T>(L);
        a.rp = L.rp;
        a.ci = L.ci;
        a.vals = level_vals<T>(L);
        a.dinv = level_dinv<T>(L);
        a.rhs = rhs;
        a.x_in = x_in;
        a.x_out = x_out;
        a.xt = L.xt;
        a.uc = uc;
        a.agg = uc ? L.agg : nullptr;
        a.field = nodef ? 0 : f;
        a.F = h->F;
        a.omega = h->p.omega;
        a.omega_node = level_omega<T>(L);
        double bytes = 0.0, flops = 0.0;
        if (h->prof && have_counts) {
            const double es = sizeof(T), B = h->b, FB = h->fb, nc = a.n_in_colour;
            const double nnz = (double)L.colour_nnz[c], low = (double)L.colour_nnz_lower[c];
            bytes = nnz * (FB * B * es + 4.0) + nc * 8.0 + nc * FB * FB * es + nc * FB * es +
                    (x_in ? nc * B * es : 0.0) + nc * B * es + nc * FB * es + (c > 0 ? nc * FB * es : 0.0) +
                    (uc ? nc * (B * es + 4.0) : 0.0);
            flops = 2.0 * ((x_in ? nnz * FB * B : 0.0) + low * FB * FB + nc * FB * FB);
        }
        if (h->rec) {
            TailPhase ph{};
            ph.type = kPhaseBgs;
            ph.n = a.n_in_colour;
            ph.bgs = a;
            record(h, ph, bytes, flops);
            continue;
        }
        PL(BAMG_K_SMOOTH, bytes, flops, launch_colour_step<T>(h, L, a, s));
    }
    if (nodef) TRY(other_fields<T>(h, L, f, x_in, x_out, uc, s));
    return BAMG_OK;
}

// transfers with the explicit (smoothed) P and R of a level, values stored
// in the cycle type or, inside an FP32 cycle, optionally in BF16
template <typename T>
static int restrict_explicit(bamg_ctx* h, const Level& L, const T* res, T* rc, cudaStream_t s);
template <>
int restrict_explicit<double>(bamg_ctx* h, const Level& L, const double* res, double* rc, cudaStream_t s) {
    return launch_fdiag_spmv<double, double>(h->b, h->fb, L.n_agg, L.r_rp, L.r_i,
                                             static_cast<const double*>(L.r_vc), res, rc, false, s);
}
template <>
int restrict_explicit<float>(bamg_ctx* h, const Level& L, const float* res, float* rc, cudaStream_t s) {
    if (h->p.pr_storage == 16)
        return launch_fdiag_spmv<float, __nv_bfloat16>(h->b, h->fb, L.n_agg, L.r_rp, L.r_i,
                                                       static_cast<const __nv_bfloat16*>(L.r_vc), res, rc, false, s);
    return launch_fdiag_spmv<float, float>(h->b, h->fb, L.n_agg, L.r_rp, L.r_i, static_cast<const float*>(L.r_vc),
                                           res, rc, false, s);
}
template <typename T>
static int prolong_explicit(bamg_ctx* h, const Level& L, const T* uc, T* u, cudaStream_t s);
template <>
int prolong_explicit<double>(bamg_ctx* h, const Level& L, const double* uc, double* u, cudaStream_t s) {
    return launch_fdiag_spmv<double, double>(h->b, h->fb, L.n, L.p_rp, L.p_ci, static_cast<const double*>(L.p_vc),
                                             uc, u, true, s);
}
template <>
int prolong_explicit<float>(bamg_ctx* h, const Level& L, const float* uc, float* u, cudaStream_t s) {
    if (h->p.pr_storage == 16)
        return launch_fdiag_spmv<float, __nv_bfloat16>(h->b, h->fb, L.n, L.p_rp, L.p_ci,
                                                       static_cast<const __nv_bfloat16*>(L.p_vc), uc, u, true, s);
    return launch_fdiag_spmv<float, float>(h->b, h->fb, L.n, L.p_rp, L.p_ci, static_cast<const float*>(L.p_vc), uc, u,
                                           true, s);
}

// the residual after the pre-smoothing can be formed from the higher-colour
// blocks alone (launch_residual_upper): one field, one sweep from zero of the
// multicolour Gauss-Seidel sub-solve (one inner sweep), one damping value for
// every node, the thread-per-row residual mapping
template <typename T>
static bool upper_residual(const bamg_ctx* h, const Level& L) {
    return h->F == 1 && h->nf <= 1 && h->p.n_pre == 1 && h->p.sub_solver == 0 && h->p.inner_sweeps <= 1 &&
           L.spmv_tpr && L.lowk && level_omega<T>(L) == nullptr;
}

// MGV(0, rhs, l) of Fig. 1 written to out
template <typename T>
static int mgv(bamg_ctx* h, int l, const T* rhs, T* out, cudaStream_t s) {
    const Level& L = h->lev[l];
    const int b = h->b;
    h->prof_level = l;  // the launches below belong to level l (until the coarser call returns)
    if (!h->rec && l == h->l_tail && h->tail_d && rhs == h->tail_rhs && out == h->tail_out) {
        // every level from l down runs as one cluster launch of the recorded phases
        if (h->tail_grid)
            PL(BAMG_K_TAIL, h->tail_bytes, h->tail_flops,
               (launch_grid_tail<T>(b, h->fb, h->tail_d, h->n_tail, h->tail_grid, h->tail_bar, h->d_err, s)));
        else
            PL(BAMG_K_TAIL, h->tail_bytes, h->tail_flops,
               launch_tail<T>(b, h->fb, h->tail_d, h->n_tail, h->tail_cluster, s));
        return BAMG_OK;
    }
    if (l == h->nlev - 1 && h->nsys > 1) {  // one dense inverse per system
        const Level& Lc = h->lev[l];
        PL(BAMG_K_COARSE, 0.0, 0.0,
           launch_batched_gemv<T>(h->nd_total, b, h->row_sys_d, Lc.sys_off_d, h->inv_off_d, h->binv, rhs, out, s));
        return BAMG_OK;
    }
    if (l == h->nlev - 1) {
        const double nd = h->nd;
        const double bytes = nd * nd * (h->coarse_inv32 ? 4.0 : 8.0) + 2.0 * nd * sizeof(T), flops = 2.0 * nd * nd;
        if (h->rec) {
            TailPhase ph{};
            ph.type = h->coarse_inv32 ? kPhaseGemv32 : kPhaseGemv;
            ph.n = h->nd;
            ph.vals = h->coarse_inv32 ? (const void*)h->coarse_inv32 : (const void*)h->coarse_inv;
            ph.x = rhs;
            ph.y = out;
            record(h, ph, bytes, flops);
            return BAMG_OK;
        }
        if (h->coarse_inv32)
            PL(BAMG_K_COARSE, bytes, flops, (launch_dense_gemv<T, float>(h->nd, h->coarse_inv32, rhs, out, s)));
        else
            PL(BAMG_K_COARSE, bytes, flops, (launch_dense_gemv<T, double>(h->nd, h->coarse_inv, rhs, out, s)));
        return BAMG_OK;
    }
    T* xa = static_cast<T*>(L.xa);
    T* xb = static_cast<T*>(L.xb);
    T* cur = nullptr;  // nullptr = the zero initial guess
    const int NS = field_steps(h);
    const int S_pre = h->p.n_pre * NS;
    for (int t = 0; t < S_pre; ++t) {
        T* dst = (cur == xa) ? xb : xa;
        TRY(bgs_step<T>(h, l, t % NS, rhs, cur, dst, nullptr, s));
        cur = dst;
    }
    if (!cur) {
        if (h->rec) {
            TailPhase ph{};
            ph.type = kPhaseZero;
            ph.n = L.n;
            ph.y = xa;
            record(h, ph, (double)L.n * b * sizeof(T), 0.0);
        } else {
            BAMG_CUDA_TRY(cudaMemsetAsync(xa, 0, sizeof(T) * (size_t)L.n * b, s));
        }
        cur = xa;
    }
    const Level& C = h->lev[l + 1];
    T* res = static_cast<T*>(L.res);
    const double es = sizeof(T), nb = (double)L.n * b, ncb = (double)C.n * b;
    if (L.smoothed) {
        // explicit transfers: r_c = R (rhs - A u), u += P u_c, then the post-smoother
        const double vs = h->p.cycle_prec == 32 && h->p.pr_storage == 16 ? 2.0 : es;
        const double tb = (double)L.p_nnz * (h->F * h->fb * h->fb * vs + 4.0);
        PL(BAMG_K_RESIDUAL, (double)L.nnzb * (b * b * es + 4.0) + (L.n + 1) * 4.0 + 3.0 * nb * es,
           2.0 * L.nnzb * b * b,
           L.spmv_tpr
               ? launch_spmv_tpr<T>(b, h->fb, level_fm<T>(L), L.n, L.rp, L.ci, level_vals<T>(L), cur, rhs, res, s)
               : launch_spmv<T>(b, h->fb, level_fm<T>(L), L.n, L.rp, L.ci, level_vals<T>(L), cur, rhs, res, s));
        PL(BAMG_K_RESTRICT, tb + (C.n + 1) * 4.0 + nb * es + ncb * es, 2.0 * L.p_nnz * b * h->fb,
           restrict_explicit<T>(h, L, res, static_cast<T*>(C.rhs), s));
        TRY(mgv<T>(h, l + 1, static_cast<const T*>(C.rhs), static_cast<T*>(C.uc), s));
        h->prof_level = l;
        PL(BAMG_K_PROLONG, tb + (L.n + 1) * 4.0 + 2.0 * nb * es + ncb * es, 2.0 * L.p_nnz * b * h->fb,
           prolong_explicit<T>(h, L, static_cast<const T*>(C.uc), cur, s));
        const int S_post = h->p.n_post * NS;
        if (S_post == 0) {
            BAMG_CUDA_TRY(cudaMemcpyAsync(out, cur, sizeof(T) * (size_t)L.n * b, cudaMemcpyDeviceToDevice, s));
            return BAMG_OK;
        }
        for (int t = 0; t < S_post; ++t) {
            T* dst = (t == S_post - 1) ? out : ((cur == xa) ? xb : xa);
            TRY(bgs_step<T>(h, l, t % NS, rhs, cur, dst, nullptr, s));
            cur = dst;
        }
        return BAMG_OK;
    }
    const double res_bytes = (double)L.nnzb * (b * b * es + 4.0) + (L.n + 1) * 4.0 + 3.0 * nb * es;
    const double res_flops = 2.0 * L.nnzb * b * b;
    const double rst_bytes = L.n * 4.0 + (C.n + 1) * 4.0 + nb * es + ncb * es;
    if (h->rec) {
        TailPhase ph{};
        ph.type = kPhaseResidual;
        ph.n = L.n;
        ph.rp = L.rp;
        ph.ci = L.ci;
        ph.vals = level_vals<T>(L);
        ph.fm = level_fm<T>(L);
        ph.x = cur;
        ph.rhs = rhs;
        ph.y = res;
        record(h, ph, res_bytes, res_flops);
        TailPhase pr{};
        pr.type = kPhaseRestrict;
        pr.n = L.n_agg;
        pr.rp = L.agg_ptr;
        pr.ci = L.members;
        pr.x = res;
        pr.y = C.rhs;
        record(h, pr, rst_bytes, nb);
    } else if (upper_residual<T>(h, L)) {
        // one sweep from zero on a one-field level: only the higher-colour blocks
        const double ub = (double)L.nnzb * 5.0 + (L.n + 1) * 4.0 + 0.5 * (L.nnzb - L.n) * (b * b * es + b * es) +
                          3.0 * nb * es;
        PL(BAMG_K_RESIDUAL, ub, (double)(L.nnzb - L.n) * b * b,
           launch_residual_upper<T>(b, level_fm<T>(L), L.n, L.rp, L.ci, L.lowk, level_vals<T>(L),
                                    static_cast<const T*>(L.xt), rhs, h->p.omega, res, s));
        PL(BAMG_K_RESTRICT, rst_bytes, nb,
           launch_restrict<T>(b, L.n_agg, L.agg_ptr, L.members, res, static_cast<T*>(C.rhs), s));
    } else {
        PL(BAMG_K_RESIDUAL, res_bytes, res_flops,
           L.spmv_tpr
               ? launch_spmv_tpr<T>(b, h->fb, level_fm<T>(L), L.n, L.rp, L.ci, level_vals<T>(L), cur, rhs, res, s)
               : launch_spmv<T>(b, h->fb, level_fm<T>(L), L.n, L.rp, L.ci, level_vals<T>(L), cur, rhs, res, s));
        PL(BAMG_K_RESTRICT, rst_bytes, nb,
           launch_restrict<T>(b, L.n_agg, L.agg_ptr, L.members, res, static_cast<T*>(C.rhs), s));
    }
    TRY(mgv<T>(h, l + 1, static_cast<const T*>(C.rhs), static_cast<T*>(C.uc), s));
    h->prof_level = l;
    const int S_post = h->p.n_post * NS;
    if (S_post == 0) {
        const double pb = L.n * 4.0 + 2.0 * nb * es + ncb * es;
        if (h->rec) {
            TailPhase ph{};
            ph.type = kPhaseProlongCopy;
            ph.n = L.n;
            ph.x = cur;
            ph.rhs = C.uc;
            ph.ci = L.agg;
            ph.y = out;
            record(h, ph, pb, nb);
        } else {
            PL(BAMG_K_PROLONG, pb, nb, launch_prolong<T>(b, L.n, L.agg, static_cast<const T*>(C.uc), cur, s));
            BAMG_CUDA_TRY(cudaMemcpyAsync(out, cur, sizeof(T) * (size_t)L.n * b, cudaMemcpyDeviceToDevice, s));
        }
    }
    // the first post-smoothing step applies u <- u + P u_c on the fly
    for (int t = 0; t < S_post; ++t) {
        T* dst = (t == S_post - 1) ? out : ((cur == xa) ? xb : xa);
        TRY(bgs_step<T>(h, l, t % NS, rhs, cur, dst, t == 0 ? static_cast<const T*>(C.uc) : nullptr, s));
        cur = dst;
    }
    return BAMG_OK;
}

// z = M r on the finest level (r, z FP64, distinct)
static int cycle_direct(bamg_ctx* h, const double* r, double* z, cudaStream_t s) {
    const long N = (long)h->lev[0].n * h->b;
    // the cycle's kernels may start while their predecessor drains (each waits
    // for its inputs); profiling keeps plain launches so that the event pairs
    // bracket one kernel each
    PdlScope pdl(h->p.use_pdl != 0 && !h->prof);
    h->prof_level = 0;
    struct OuterLevel {  // launches after the cycle belong to the outer method
        bamg_ctx* h;
        ~OuterLevel() { h->prof_level = -1; }
    } outer_level{h};
    if (h->p.cycle_prec == 64) {
        if (h->tail_d && h->l_tail == 0 && (r != h->cyc_in || z != h->cyc_out)) {
            // the recorded single-launch cycle reads and writes the staging vectors
            BAMG_CUDA_TRY(cudaMemcpyAsync(h->cyc_in, r, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
            TRY(mgv<double>(h, 0, h->cyc_in, h->cyc_out, s));
            BAMG_CUDA_TRY(cudaMemcpyAsync(z, h->cyc_out, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
            return BAMG_OK;
        }
        return mgv<double>(h, 0, r, z, s);
    }
    PL(BAMG_K_CAST, N * 12.0, 0.0, launch_cast_d2f(N, r, h->r32, s));
    TRY(mgv<float>(h, 0, h->r32, h->z32, s));
    PL(BAMG_K_CAST, N * 12.0, 0.0, launch_cast_f2d(N, h->z32, z, s));
    return BAMG_OK;
}

// Record the phases of every level from l_tail down (device copy in tail_d).
// With only_counts the phases are recorded to refresh the byte / flop totals.
static int record_tail(bamg_ctx* h, cudaStream_t s, bool only_counts) {
    std::vector<TailPhase> phases;
    h->rec = &phases;
    h->rec_bytes = h->rec_flops = 0.0;
    const int lt = h->l_tail;
    int st;
    if (h->p.cycle_prec == 64) {
        const double* rhs = lt == 0 ? h->cyc_in : static_cast<const double*>(h->lev[lt].rhs);
        double* out = lt == 0 ? h->cyc_out : static_cast<double*>(h->lev[lt].uc);
        h->tail_rhs = rhs;
        h->tail_out = out;
        st = mgv<double>(h, lt, rhs, out, s);
    } else {
        const float* rhs = lt == 0 ? h->r32 : static_cast<const float*>(h->lev[lt].rhs);
        float* out = lt == 0 ? h->z32 : static_cast<float*>(h->lev[lt].uc);
        h->tail_rhs = rhs;
        h->tail_out = out;
        st = mgv<float>(h, lt, rhs, out, s);
    }
    h->rec = nullptr;
    if (st != BAMG_OK) return st;
    h->tail_bytes = h->rec_bytes;
    h->tail_flops = h->rec_flops;
    if (only_counts) return BAMG_OK;
    TailPhase* d = nullptr;
    TRY(h->alloc(&d, phases.size()));
    BAMG_CUDA_TRY(cudaMemcpyAsync(d, phases.data(), sizeof(TailPhase) * phases.size(), cudaMemcpyHostToDevice, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    h->n_tail = (int)phases.size();
    h->tail_d = d;
    return BAMG_OK;
}

// choose the first level of the cluster tail and record its phases
static int setup_tail(bamg_ctx* h, cudaStream_t s) {
    h->tail_d = nullptr;
    h->l_tail = -1;
    if (h->p.tail_dofs <= 0 || h->nlev < 2) return BAMG_OK;
    for (int l = 0; l + 1 < h->nlev; ++l)
        if (h->lev[l].smoothed) return BAMG_OK;  // the tail kernel has no explicit-transfer phase
    int lt = h->nlev - 1;
    while (lt > 0 && (long)h->lev[lt - 1].n * h->b <= h->p.tail_dofs) --lt;
    if (lt >= h->nlev - 1) return BAMG_OK;  // only the coarsest solve would remain: no gain
    if (h->p.tail_grid) {
        const int g = h->p.cycle_prec == 64 ? grid_tail_size<double>(h->b, h->fb) : grid_tail_size<float>(h->b, h->fb);
        if (g < 1) return BAMG_OK;  // no cooperative launch: per-kernel cycle
        TRY(h->alloc(&h->tail_bar, 2));
        BAMG_CUDA_TRY(cudaMemsetAsync(h->tail_bar, 0, 2 * sizeof(unsigned), s));
        h->tail_grid = g;
    } else {
        const int cl = h->p.cycle_prec == 64 ? tail_cluster_size<double>(h->b, h->fb, 16)
                                             : tail_cluster_size<float>(h->b, h->fb, 16);
        if (cl < 1) return BAMG_OK;
        h->tail_cluster = cl;
    }
    h->l_tail = lt;
    return record_tail(h, s, false);
}

static int ensure_graph(bamg_ctx* h) {
    if (h->graph_exec) return BAMG_OK;
    cudaStream_t cs = h->cap_stream;
    BAMG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    long long kernels = 0;
    t_capture_sink = &kernels;
    int st = cycle_direct(h, h->cyc_in, h->cyc_out, cs);
    t_capture_sink = nullptr;
    h->graph_kernels = kernels;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (st != BAMG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return BAMG_ECUDA;
    h->graph = g;
    BAMG_CUDA_TRY(cudaGraphInstantiate(&h->graph_exec, g, 0));
    return BAMG_OK;
}

// the V-cycle captured with an event-record node around every kernel
static int ensure_prof_graph(bamg_ctx* h) {
    if (h->prof_exec) return BAMG_OK;
    cudaStream_t cs = h->cap_stream;
    BAMG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    long long kernels = 0;
    t_capture_sink = &kernels;
    h->capturing_prof = true;
    int st = cycle_direct(h, h->cyc_in, h->cyc_out, cs);
    h->capturing_prof = false;
    t_capture_sink = nullptr;
    h->prof_graph_kernels = kernels;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (st != BAMG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return BAMG_ECUDA;
    h->prof_graph = g;
    BAMG_CUDA_TRY(cudaGraphInstantiate(&h->prof_exec, g, 0));
    return BAMG_OK;
}

static int apply_profiled(bamg_ctx* h, const double* r, double* z, cudaStream_t s) {
    TRY(ensure_prof_graph(h));
    const size_t nbytes = sizeof(double) * (size_t)h->lev[0].n * h->b;
    BAMG_CUDA_TRY(cudaMemcpyAsync(h->cyc_in, r, nbytes, cudaMemcpyDeviceToDevice, s));
    BAMG_CUDA_TRY(cudaGraphLaunch(h->prof_exec, s));
    note_launch((int)h->prof_graph_kernels);
    BAMG_CUDA_TRY(cudaMemcpyAsync(z, h->cyc_out, nbytes, cudaMemcpyDeviceToDevice, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    for (const ProfRec& rec : h->graph_recs) {
        float e = 0.0f;
        BAMG_CUDA_TRY(cudaEventElapsedTime(&e, rec.e0, rec.e1));
        const int sl = rec.level + 1;
        h->acc_ms[rec.kind][sl] += e;
        h->acc_bytes[rec.kind][sl] += rec.bytes;
        h->acc_flops[rec.kind][sl] += rec.flops;
        h->acc_n[rec.kind][sl] += 1;
    }
    return BAMG_OK;
}

static int apply_impl(bamg_ctx* h, const double* r, double* z, cudaStream_t s) {
    if (h->prof && h->p.use_graph) return apply_profiled(h, r, z, s);
    // (a cycle with the cooperative grid tail is one launch plus casts: direct)
    if (!h->p.use_graph || h->prof || h->tail_grid) return cycle_direct(h, r, z, s);
    TRY(ensure_graph(h));
    const size_t nbytes = sizeof(double) * (size_t)h->lev[0].n * h->b;
    BAMG_CUDA_TRY(cudaMemcpyAsync(h->cyc_in, r, nbytes, cudaMemcpyDeviceToDevice, s));
    BAMG_CUDA_TRY(cudaGraphLaunch(h->graph_exec, s));
    note_launch((int)h->graph_kernels);
    BAMG_CUDA_TRY(cudaMemcpyAsync(z, h->cyc_out, nbytes, cudaMemcpyDeviceToDevice, s));
    return BAMG_OK;
}

extern "C" int amg_apply(bamg_t h, const double* r, double* z, void* stream) {
    if (!h || !r || !z || r == z) return BAMG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (h->padded) {  // fields of unequal size: the cycle of the padded system
        const long n = h->lev[0].n;
        TRY(launch_pad_vec(h->pad, n, r, h->pad_b, s));
        TRY(apply_impl(h, h->pad_b, h->pad_x, s));
        return launch_unpad_vec(h->pad, n, h->pad_x, z, s);
    }
    return apply_impl(h, r, z, s);
}

// the solve of a padded hierarchy (fields of unequal size): b and x padded
// into the handle's vectors, the solve on them, x unpadded
template <class Solve>
static int padded_solve(bamg_ctx* h, const double* b, double* x, cudaStream_t s, Solve&& solve) {
    const long n = h->lev[0].n;
    TRY(launch_pad_vec(h->pad, n, b, h->pad_b, s));
    TRY(launch_pad_vec(h->pad, n, x, h->pad_x, s));
    const int st = solve(h->pad_b, h->pad_x);
    if (st < 0) return st;
    TRY(launch_unpad_vec(h->pad, n, h->pad_x, x, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    return st;
}

// ---------------------------------------------------------------------------
// FGMRES
// ---------------------------------------------------------------------------
static int ensure_krylov(bamg_ctx* h, int m) {
    if (h->m_alloc >= m) return BAMG_OK;
    for (void* q : {(void*)h->V, (void*)h->Z, (void*)h->w, (void*)h->partial, (void*)h->h1, (void*)h->h2,
                    (void*)h->wsq, (void*)h->H, (void*)h->cs, (void*)h->sn, (void*)h->g, (void*)h->y,
                    (void*)h->scal, (void*)h->ticket})
        if (q) h->release(q);
    const size_t N = (size_t)h->lev[0].n * h->b;
    const int nchunk = krylov_chunks((long)N);
    TRY(h->alloc(&h->V, N * (m + 1)));
    TRY(h->alloc(&h->Z, N * m));
    TRY(h->alloc(&h->w, N));
    TRY(h->alloc(&h->partial, (size_t)(m + 2) * nchunk));
    TRY(h->alloc(&h->h1, (size_t)m + 2));
    TRY(h->alloc(&h->h2, (size_t)m + 2));
    TRY(h->alloc(&h->wsq, 2));
    TRY(h->alloc(&h->H, (size_t)(m + 1) * m));
    TRY(h->alloc(&h->cs, (size_t)m));
    TRY(h->alloc(&h->sn, (size_t)m));
    TRY(h->alloc(&h->g, (size_t)m + 1));
    TRY(h->alloc(&h->y, (size_t)m));
    TRY(h->alloc(&h->scal, 4));
    TRY(h->alloc(&h->ticket, 4));
    BAMG_CUDA_TRY(cudaMemsetAsync(h->ticket, 0, 4 * sizeof(unsigned), h->stream));
    BAMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->m_alloc = m;
    return BAMG_OK;
}

// y = A x (or rhs - A x) with the finest FP64 operator, in the tuned row mapping
static int outer_spmv(bamg_ctx* h, const double* x, const double* rhs, double* y, cudaStream_t s) {
    const Level& L0 = h->lev[0];
    return h->outer_spmv_tpr ? launch_spmv_tpr<double>(h->b, h->fb, 0, L0.n, L0.rp, L0.ci, L0.vals64, x, rhs, y, s,
                                                       h->outer_spmv_tpr - 1)
                             : launch_spmv<double>(h->b, h->fb, 0, L0.n, L0.rp, L0.ci, L0.vals64, x, rhs, y, s);
}

// ||x||^2 into dst (device), via the deterministic chunked reduction
static int norm_sq(bamg_ctx* h, long N, const double* x, double* dst, cudaStream_t s) {
    PL(BAMG_K_KRYLOV, N * 8.0, 2.0 * N, launch_multi_dot(N, x, nullptr, 0, 0, 1, h->partial, dst, h->ticket, s));
    return BAMG_OK;
}

static int fgmres_impl(bamg_t h, const double* b, double* x, double tol, int restart, int max_iter, int* iters,
                       double* relres, void* stream);

extern "C" int fgmres_solve(bamg_t h, const double* b, double* x, double tol, int restart, int max_iter,
                            int* iters, double* relres, void* stream) {
    if (!h || !b || !x || restart < 1 || restart > kMaxRestart || max_iter < 0 || !(tol >= 0.0))
        return BAMG_EINVAL;
    if (h->padded)
        return padded_solve(h, b, x, static_cast<cudaStream_t>(stream), [&](const double* bp, double* xp) {
            return fgmres_impl(h, bp, xp, tol, restart, max_iter, iters, relres, stream);
        });
    return fgmres_impl(h, b, x, tol, restart, max_iter, iters, relres, stream);
}

static int fgmres_impl(bamg_t h, const double* b, double* x, double tol, int restart, int max_iter, int* iters,
                       double* relres, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int m = restart;
    TRY(ensure_krylov(h, m));
    h->arnoldi_steps = 0;
    h->second_projections = 0;
    const Level& L0 = h->lev[0];
    const long N = (long)L0.n * h->b;
    const int bsz = h->b;
    double* hs = h->h_scal;
    TRY(norm_sq(h, N, b, h->wsq, s));
    BAMG_CUDA_TRY(cudaMemcpyAsync(hs, h->wsq, sizeof(double), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    const double bnorm = sqrt(hs[0]);
    if (!isfinite(bnorm)) return BAMG_ENAN;
    int total = 0, converged = 0;
    double rel = 0.0;
    if (bnorm == 0.0) {
        BAMG_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        converged = 1;
    }
    const double spmv_bytes = (double)L0.nnzb * (bsz * bsz * 8.0 + 4.0) + (L0.n + 1) * 4.0 + 2.0 * N * 8.0;
    const double spmv_flops = 2.0 * L0.nnzb * bsz * bsz;
    const double vN = N * 8.0;
    while (!converged) {
        PL(BAMG_K_SPMV, spmv_bytes + vN, spmv_flops,
           outer_spmv(h, x, b, h->w, s));  // w = b - A x
        TRY(norm_sq(h, N, h->w, h->wsq, s));
        BAMG_CUDA_TRY(cudaMemcpyAsync(hs, h->wsq, sizeof(double), cudaMemcpyDeviceToHost, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        const double beta = sqrt(hs[0]);
        rel = beta / bnorm;
        if (!isfinite(rel)) return BAMG_ENAN;
        if (rel <= tol) {
            converged = 1;
            break;
        }
        if (total >= max_iter) break;
        PL(BAMG_K_KRYLOV, 0.0, 0.0, launch_init_g(m, h->wsq, h->g, h->scal, s));
        PL(BAMG_K_KRYLOV, 2.0 * vN, N, launch_scale(N, h->w, h->scal, h->V, 0, s));  // v_0 = r / beta
        int k = 0;
        for (int j = 0; j < m; ++j) {
            const double* vj = h->V + (size_t)j * N;
            double* zj = h->Z + (size_t)j * N;
            TRY(apply_impl(h, vj, zj, s));
            PL(BAMG_K_SPMV, spmv_bytes, spmv_flops,
               outer_spmv(h, zj, nullptr, h->w, s));
            const double nv = j + 1;
            GivensArgs ga{j, m, h->h1, h->h2, h->H, h->cs, h->sn, h->g, h->scal};
            PL(BAMG_K_KRYLOV, (nv + 1) * vN, 2.0 * N * (nv + 1),
               launch_multi_dot(N, h->w, h->V, N, j + 1, 1, h->partial, h->h1, h->ticket, s));
            if (h->p.ortho == 1) {
                // CGS2: h1 = V^T w (and ||w||^2), w -= V h1, h2 = V^T w, w -= V h2, ||w||^2
                PL(BAMG_K_KRYLOV, (2 * nv + 2) * vN, 4.0 * N * nv,
                   launch_axpy_dot(N, h->w, h->V, N, j + 1, h->h1, 1.0, 1, h->partial, h->h2, h->ticket, nullptr,
                                   s));
                PL(BAMG_K_KRYLOV, (nv + 2) * vN, 2.0 * N * (nv + 1),
                   launch_axpy_dot(N, h->w, h->V, N, j + 1, h->h2, 1.0, 2, h->partial, h->wsq, h->ticket, &ga, s));
            } else {
                // classical Gram-Schmidt, projected a second time only where the
                // norm of w left after the first projection is below 0.01 of the
                // norm before it (the selective test of Daniel, Gragg, Kaufman and
                // Stewart): w -= V h1 and ||w||^2 with the test; then, only if
                // set, h2 = V^T w and w -= V h2, ||w||^2 (Givens with h1 + h2)
                unsigned* reorth = h->ticket + 2;
                PL(BAMG_K_KRYLOV, (nv + 2) * vN, 2.0 * N * (nv + 1),
                   launch_axpy_dot(N, h->w, h->V, N, j + 1, h->h1, 1.0, 3, h->partial, h->wsq, h->ticket, &ga, s,
                                   nullptr, reorth));
                PL(BAMG_K_KRYLOV, 0.0, 0.0,
                   launch_multi_dot(N, h->w, h->V, N, j + 1, 0, h->partial, h->h2, h->ticket, s, reorth));
                PL(BAMG_K_KRYLOV, 0.0, 0.0,
                   launch_axpy_dot(N, h->w, h->V, N, j + 1, h->h2, 1.0, 2, h->partial, h->wsq, h->ticket, &ga, s,
                                   reorth));
            }
            PL(BAMG_K_KRYLOV, 2.0 * vN, N, launch_scale(N, h->w, h->scal, h->V + (size_t)(j + 1) * N, 1, s));
            total++;
            h->arnoldi_steps++;
            k = j + 1;
            BAMG_CUDA_TRY(cudaMemcpyAsync(hs, h->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
            // a bounded wait of the cycle (grid barrier, sweep tile) that ran out
            BAMG_CUDA_TRY(cudaMemcpyAsync(h->h_pin, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
            if (h->p.ortho != 1)  // whether this step projected twice (statistics)
                BAMG_CUDA_TRY(cudaMemcpyAsync(h->h_pin + 5, h->ticket + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
            BAMG_CUDA_TRY(cudaStreamSynchronize(s));
            if (h->h_pin[0] != 0) return map_dev_error(h->h_pin[0]);
            h->second_projections += h->p.ortho == 1 ? 1 : (h->h_pin[5] != 0 ? 1 : 0);
            if (!isfinite(hs[1])) return BAMG_ENAN;
            if (hs[1] / bnorm <= tol || hs[2] != 0.0 || total >= max_iter) break;
        }
        PL(BAMG_K_KRYLOV, 0.0, 0.0, launch_solve_upper(k, m, h->H, h->g, h->y, s));
        PL(BAMG_K_KRYLOV, (k + 2.0) * vN, 2.0 * N * k,
           launch_axpy_dot(N, x, h->Z, N, k, h->y, -1.0, 0, nullptr, nullptr, h->ticket, nullptr, s));  // x += Z y
    }
    if (iters) *iters = total;
    if (relres) *relres = rel;
    return converged ? BAMG_OK : BAMG_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// FGMRES for a batch: every system runs its own FGMRES(m) (own Krylov basis,
// Hessenberg matrix, rotations, stopping test and iteration count); the
// V-cycle and the SpMV act on all systems at once, reductions are per system.
// ---------------------------------------------------------------------------
static int ensure_batched_krylov(bamg_ctx* h, int m) {
    if (h->mb_alloc >= m) return BAMG_OK;
    for (void* q : {(void*)h->bh1, (void*)h->bh2, (void*)h->bwsq, (void*)h->bH, (void*)h->bcs, (void*)h->bsn,
                    (void*)h->bg, (void*)h->by, (void*)h->bscal, (void*)h->bsq, (void*)h->bk, (void*)h->bactive,
                    (void*)h->bincycle})
        if (q) h->release(q);
    const size_t S = (size_t)h->nsys;
    TRY(h->alloc(&h->bh1, S * (m + 2)));
    TRY(h->alloc(&h->bh2, S * (m + 2)));
    TRY(h->alloc(&h->bwsq, S));
    TRY(h->alloc(&h->bH, S * (m + 1) * m));
    TRY(h->alloc(&h->bcs, S * m));
    TRY(h->alloc(&h->bsn, S * m));
    TRY(h->alloc(&h->bg, S * (m + 1)));
    TRY(h->alloc(&h->by, S * m));
    TRY(h->alloc(&h->bscal, S * 4));
    TRY(h->alloc(&h->bsq, S));
    TRY(h->alloc(&h->bk, S));
    TRY(h->alloc(&h->bactive, S));
    TRY(h->alloc(&h->bincycle, S));
    h->hb_scal.assign(S * 4, 0.0);
    BAMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->mb_alloc = m;
    return BAMG_OK;
}

static int fgmres_batched_impl(bamg_t h, const double* b, double* x, double tol, int restart, int max_iter,
                               int* iters, double* relres, void* stream);

extern "C" int fgmres_solve_batched(bamg_t h, const double* b, double* x, double tol, int restart, int max_iter,
                                    int* iters, double* relres, void* stream) {
    if (!h || !b || !x || restart < 1 || restart > kMaxRestart || max_iter < 0 || !(tol >= 0.0)) return BAMG_EINVAL;
    if (h->padded)
        return padded_solve(h, b, x, static_cast<cudaStream_t>(stream), [&](const double* bp, double* xp) {
            return fgmres_batched_impl(h, bp, xp, tol, restart, max_iter, iters, relres, stream);
        });
    return fgmres_batched_impl(h, b, x, tol, restart, max_iter, iters, relres, stream);
}

static int fgmres_batched_impl(bamg_t h, const double* b, double* x, double tol, int restart, int max_iter,
                               int* iters, double* relres, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int m = restart, S = h->nsys;
    TRY(ensure_krylov(h, m));
    TRY(ensure_batched_krylov(h, m));
    if (h->m_alloc == m)  // a fresh basis: keep unused systems' chunks finite
        BAMG_CUDA_TRY(cudaMemsetAsync(h->V, 0, sizeof(double) * (size_t)h->lev[0].n * h->b * (m + 1), s));
    const Level& L0 = h->lev[0];
    const long N = (long)L0.n * h->b;
    const int bsz = h->b;
    const SegTable& T = h->seg;
    double* partial = nullptr;
    TRY(h->alloc(&partial, (size_t)(m + 2) * T.nchunk));
    BAMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    std::vector<double> bn((size_t)S), rel((size_t)S, 0.0), tmp((size_t)S);
    std::vector<int> conv((size_t)S, 0), tot((size_t)S, 0), active((size_t)S), incycle((size_t)S), kk((size_t)S);
    auto download = [&](const double* d, double* hp, size_t cnt) -> int {
        BAMG_CUDA_TRY(cudaMemcpyAsync(hp, d, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        return BAMG_OK;
    };
    auto upload = [&](int* d, const std::vector<int>& v) -> int {
        BAMG_CUDA_TRY(cudaMemcpyAsync(d, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, s));
        return BAMG_OK;
    };
    // ||b_s||
    TRY(launch_seg_dots(T, b, nullptr, 0, 0, 1, partial, h->bsq, 1, s));
    TRY(download(h->bsq, tmp.data(), (size_t)S));
    for (int q = 0; q < S; ++q) {
        bn[q] = sqrt(tmp[q]);
        if (!std::isfinite(bn[q])) {
            h->release(partial);
            return BAMG_ENAN;
        }
        if (bn[q] == 0.0) {  // x_s = 0 solves it
            conv[q] = 1;
            const size_t e0 = (size_t)L0.sys_off[q] * bsz, e1 = (size_t)L0.sys_off[q + 1] * bsz;
            BAMG_CUDA_TRY(cudaMemsetAsync(x + e0, 0, sizeof(double) * (e1 - e0), s));
        }
    }
    int st = BAMG_OK;
    for (;;) {
        TRY(outer_spmv(h, x, b, h->w, s));  // w = b - A x
        TRY(launch_seg_dots(T, h->w, nullptr, 0, 0, 1, partial, h->bsq, 1, s));
        TRY(download(h->bsq, tmp.data(), (size_t)S));
        int n_active = 0;
        for (int q = 0; q < S; ++q) {
            if (bn[q] == 0.0) continue;
            rel[q] = sqrt(tmp[q]) / bn[q];
            if (!std::isfinite(rel[q])) st = BAMG_ENAN;
            if (rel[q] <= tol) conv[q] = 1;
            active[q] = !conv[q] && tot[q] < max_iter;
            incycle[q] = active[q];
            kk[q] = 0;
            n_active += active[q];
        }
        for (int q = 0; q < S; ++q)
            if (bn[q] == 0.0) active[q] = incycle[q] = kk[q] = 0;
        if (st != BAMG_OK || n_active == 0) break;
        TRY(upload(h->bactive, active));
        TRY(upload(h->bincycle, incycle));
        TRY(launch_seg_init_g(S, m, h->bsq, h->bg, h->bscal, s));
        TRY(launch_seg_scale(T, h->w, h->bscal, h->V, h->bactive, 0, s));  // v_0 = r / beta per system
        for (int j = 0; j < m; ++j) {
            const double* vj = h->V + (size_t)j * N;
            double* zj = h->Z + (size_t)j * N;
            TRY(apply_impl(h, vj, zj, s));
            TRY(outer_spmv(h, zj, nullptr, h->w, s));
            TRY(launch_seg_dots(T, h->w, h->V, N, j + 1, 1, partial, h->bh1, m + 2, s));
            TRY(launch_seg_axpy_dots(T, h->w, h->V, N, j + 1, h->bh1, m + 2, 1.0, 1, h->bincycle, partial, h->bh2,
                                     m + 2, s));
            TRY(launch_seg_axpy_dots(T, h->w, h->V, N, j + 1, h->bh2, m + 2, 1.0, 2, h->bincycle, partial, h->bwsq,
                                     1, s));
            TRY(launch_seg_givens(S, j, m, h->bh1, h->bh2, h->bwsq, h->bH, h->bcs, h->bsn, h->bg, h->bscal,
                                  h->bincycle, s));
            TRY(launch_seg_scale(T, h->w, h->bscal, h->V + (size_t)(j + 1) * N, h->bincycle, 1, s));
            TRY(download(h->bscal, h->hb_scal.data(), (size_t)S * 4));
            int left = 0;
            for (int q = 0; q < S; ++q) {
                if (!incycle[q]) continue;
                kk[q] = j + 1;
                tot[q]++;
                const double est = h->hb_scal[(size_t)q * 4 + 1];
                if (!std::isfinite(est)) st = BAMG_ENAN;
                if (est / bn[q] <= tol || h->hb_scal[(size_t)q * 4 + 2] != 0.0 || tot[q] >= max_iter) incycle[q] = 0;
                left += incycle[q];
            }
            if (st != BAMG_OK || left == 0) break;
            TRY(upload(h->bincycle, incycle));
        }
        if (st != BAMG_OK) break;
        TRY(upload(h->bk, kk));
        TRY(launch_seg_solve_upper(S, m, h->bk, h->bH, h->bg, h->by, s));
        TRY(launch_seg_axpy_dots(T, x, h->Z, N, m, h->by, m, -1.0, 0, h->bactive, nullptr, nullptr, 0, s));  // x += Z y
    }
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    h->release(partial);
    if (st == BAMG_OK) {  // a bounded wait of the cycle (sweep tile) that ran out
        const int dev_st = check_dev(h, s);
        if (dev_st != BAMG_OK) return dev_st;
    }
    int all = 1;
    for (int q = 0; q < S; ++q) {
        if (iters) iters[q] = tot[q];
        if (relres) relres[q] = rel[q];
        all &= conv[q];
    }
    if (st != BAMG_OK) return st;
    return all ? BAMG_OK : BAMG_NOT_CONVERGED;
}

extern "C" int amg_num_systems(bamg_t h) { return h ? h->nsys : BAMG_EINVAL; }

extern "C" int amg_level_systems(bamg_t h, int level, int* sys_node_off) {
    if (!h || level < 0 || level >= h->nlev || !sys_node_off) return BAMG_EINVAL;
    const Level& L = h->lev[level];
    for (size_t q = 0; q < L.sys_off.size(); ++q) sys_node_off[q] = L.sys_off[q];
    return BAMG_OK;
}

// ---------------------------------------------------------------------------
// end-to-end with host buffers
// ---------------------------------------------------------------------------
// End to end with host buffers: copies of the pattern, b and x0 on the device
// (the stream-ordered pool), setup(d_rp, d_ci, vals, &h) with the HOST values
// (the setup copies them into its own level-0 array on a side stream while its
// pattern phases run) and solve(h, d_b, d_x), x back to the host, everything
// released.
template <class Setup, class Solve>
static int solve_host_common(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int nnzb,
                             int b, const double* rhs_host, double* x_host, void* stream, Setup&& setup,
                             Solve&& solve) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t N = (size_t)n_nodes * b;
    int *d_rp = nullptr, *d_ci = nullptr;
    double *d_b = nullptr, *d_x = nullptr;
    int st = BAMG_OK;
    bamg_t h = nullptr;
    if (pool_alloc((void**)&d_rp, sizeof(int) * (n_nodes + 1), s) != cudaSuccess ||
        pool_alloc((void**)&d_ci, sizeof(int) * (size_t)nnzb, s) != cudaSuccess ||
        pool_alloc((void**)&d_b, sizeof(double) * N, s) != cudaSuccess ||
        pool_alloc((void**)&d_x, sizeof(double) * N, s) != cudaSuccess)
        st = BAMG_ECUDA;
    if (st == BAMG_OK &&
        (cudaMemcpyAsync(d_rp, row_ptr, sizeof(int) * (n_nodes + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(d_ci, col_idx, sizeof(int) * (size_t)nnzb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(d_b, rhs_host, sizeof(double) * N, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(d_x, x_host, sizeof(double) * N, cudaMemcpyHostToDevice, s) != cudaSuccess))
        st = BAMG_ECUDA;
    if (st == BAMG_OK) st = setup(d_rp, d_ci, vals, &h);
    int solve_st = BAMG_OK;
    if (st == BAMG_OK) {
        solve_st = solve(h, d_b, d_x);
        if (solve_st >= 0 &&
            (cudaMemcpyAsync(x_host, d_x, sizeof(double) * N, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess))
            solve_st = BAMG_ECUDA;
    }
    cudaStreamSynchronize(s);
    amg_destroy(h);
    for (void* q : {(void*)d_rp, (void*)d_ci, (void*)d_b, (void*)d_x})
        if (q) cudaFreeAsync(q, s);
    cudaStreamSynchronize(s);
    return st != BAMG_OK ? st : solve_st;
}

extern "C" int amg_solve_host(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes,
                              int nnzb, int b, const int* field_of_dof, const amg_params* p,
                              const double* rhs_host, double* x_host, double tol, int restart, int max_iter,
                              int* iters, double* relres, void* stream) {
    if (!row_ptr || !col_idx || !vals || !rhs_host || !x_host || n_nodes < 1 || nnzb < 1 || b < 1 || b > kMaxB)
        return BAMG_EINVAL;
    return solve_host_common(
        row_ptr, col_idx, vals, n_nodes, nnzb, b, rhs_host, x_host, stream,
        [&](const int* rp, const int* ci, const double* v, bamg_t* h) {
            return setup_common(rp, ci, v, n_nodes, nnzb, b, field_of_dof, p, stream, h, 1, nullptr, 1, nullptr,
                                true);
        },
        [&](bamg_t h, const double* bb, double* x) {
            return fgmres_solve(h, bb, x, tol, restart, max_iter, iters, relres, stream);
        });
}

extern "C" int amg_solve_batched_host(int nsys, const int* sys_node_off, const int* row_ptr, const int* col_idx,
                                      const double* vals, int n_nodes, int nnzb, int b, const int* field_of_dof,
                                      const amg_params* p, const double* rhs_host, double* x_host, double tol,
                                      int restart, int max_iter, int* iters, double* relres, void* stream) {
    if (nsys < 1 || !sys_node_off || !row_ptr || !col_idx || !vals || !rhs_host || !x_host || n_nodes < 1 ||
        nnzb < 1 || b < 1 || b > kMaxB)
        return BAMG_EINVAL;
    return solve_host_common(
        row_ptr, col_idx, vals, n_nodes, nnzb, b, rhs_host, x_host, stream,
        [&](const int* rp, const int* ci, const double* v, bamg_t* h) {
            return setup_common(rp, ci, v, n_nodes, nnzb, b, field_of_dof, p, stream, h, nsys, sys_node_off, 1,
                                nullptr, true);
        },
        [&](bamg_t h, const double* bb, double* x) {
            return fgmres_solve_batched(h, bb, x, tol, restart, max_iter, iters, relres, stream);
        });
}

extern "C" int amg_solve_fields_host(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes,
                                     int nnzb, int b, int n_fields, const int* field_node_off, const amg_params* p,
                                     const double* rhs_host, double* x_host, double tol, int restart, int max_iter,
                                     int* iters, double* relres, void* stream) {
    if (!row_ptr || !col_idx || !vals || !rhs_host || !x_host || !field_node_off || n_nodes < 1 || nnzb < 1 ||
        b < 1 || b > kMaxB || n_fields < 1)
        return BAMG_EINVAL;
    return solve_host_common(
        row_ptr, col_idx, vals, n_nodes, nnzb, b, rhs_host, x_host, stream,
        [&](const int* rp, const int* ci, const double* v, bamg_t* h) {
            return setup_fields(rp, ci, v, n_nodes, nnzb, b, n_fields, field_node_off, p, stream, h, true);
        },
        [&](bamg_t h, const double* bb, double* x) {
            return fgmres_solve(h, bb, x, tol, restart, max_iter, iters, relres, stream);
        });
}

// ---------------------------------------------------------------------------
// plain SpMV entry point
// ---------------------------------------------------------------------------
extern "C" int bsr_spmv(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int b,
                        const double* x, double* y, void* stream) {
    if (!row_ptr || !col_idx || !vals || !x || !y || n_nodes < 0 || b < 1 || b > kMaxB || x == y)
        return BAMG_EINVAL;
    return launch_spmv<double>(b, b, 0, n_nodes, row_ptr, col_idx, vals, x, nullptr, y,
                               static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// introspection
// ---------------------------------------------------------------------------
extern "C" int amg_num_levels(bamg_t h) { return h ? h->nlev : BAMG_EINVAL; }

extern "C" int amg_block_size(bamg_t h) { return h ? h->b : BAMG_EINVAL; }

extern "C" int amg_level_info(bamg_t h, int level, int* n_nodes, int* nnzb, int* n_colours, int* n_agg) {
    if (!h || level < 0 || level >= h->nlev) return BAMG_EINVAL;
    const Level& L = h->lev[level];
    const bool coarsest = level == h->nlev - 1;
    if (n_nodes) *n_nodes = L.n;
    if (nnzb) *nnzb = L.nnzb;
    if (n_colours) *n_colours = coarsest ? 0 : L.n_colours;
    if (n_agg) *n_agg = coarsest ? 0 : L.n_agg;
    return BAMG_OK;
}

extern "C" int amg_level_copy(bamg_t h, int level, int* row_ptr, int* col_idx, double* vals, int* agg,
                              int* colour, double* dinv) {
    if (!h || level < 0 || level >= h->nlev) return BAMG_EINVAL;
    const Level& L = h->lev[level];
    const bool coarsest = level == h->nlev - 1;
    const size_t bb = (size_t)h->b * h->b;
    if (row_ptr) BAMG_CUDA_TRY(cudaMemcpy(row_ptr, L.rp, sizeof(int) * (L.n + 1), cudaMemcpyDefault));
    if (col_idx) BAMG_CUDA_TRY(cudaMemcpy(col_idx, L.ci, sizeof(int) * (size_t)L.nnzb, cudaMemcpyDefault));
    if (vals) BAMG_CUDA_TRY(cudaMemcpy(vals, L.vals64, sizeof(double) * bb * L.nnzb, cudaMemcpyDefault));
    if (!coarsest) {
        if (agg) BAMG_CUDA_TRY(cudaMemcpy(agg, L.agg, sizeof(int) * (size_t)L.n, cudaMemcpyDefault));
        if (colour) BAMG_CUDA_TRY(cudaMemcpy(colour, L.colour, sizeof(int) * (size_t)L.n, cudaMemcpyDefault));
        if (dinv)
            BAMG_CUDA_TRY(cudaMemcpy(dinv, L.dinv64, sizeof(double) * (size_t)L.n * h->F * h->fb * h->fb,
                                     cudaMemcpyDefault));
    }
    return BAMG_OK;
}

extern "C" int amg_level_ilu(bamg_t h, int level, double* lu) {
    if (!h || level < 0 || level >= h->nlev || !lu) return BAMG_EINVAL;
    const Level& L = h->lev[level];
    if (!L.ilu64) return BAMG_EINVAL;
    BAMG_CUDA_TRY(cudaMemcpy(lu, L.ilu64, sizeof(double) * (size_t)h->F * L.nnzb * h->fb * h->fb,
                             cudaMemcpyDefault));
    return BAMG_OK;
}

extern "C" int amg_stats(bamg_t h, char* json, int cap) {
    if (!h || !json || cap < 1) return BAMG_EINVAL;
    std::string o = "{\"b\":" + std::to_string(h->b) + ",\"b_given\":" + std::to_string(h->padded ? h->pad.b : h->b) +
                    ",\"padded\":" + std::to_string(h->padded ? 1 : 0) + ",\"fields\":" + std::to_string(h->F) +
                    ",\"node_fields\":" + std::to_string(h->nf) + ",\"cycle_prec\":" + std::to_string(h->p.cycle_prec) +
                    ",\"coarse_prec\":" + std::to_string(h->coarse_inv32 ? 32 : 64) + ",\"coarse_tc\":" + std::to_string(h->coarse_tc_used ? 1 : 0) + ",\"arnoldi_steps\":" + std::to_string(h->arnoldi_steps) + ",\"second_projections\":" + std::to_string(h->second_projections) + ",\"sub_solver\":" + std::to_string(h->p.sub_solver) + ",\"inner_sweeps\":" + std::to_string(h->p.inner_sweeps) + ",\"outer_mapping\":\"" + (h->outer_spmv_tpr == 2 ? "thread-split" : h->outer_spmv_tpr ? "thread" : "warp") + "\",\"outer_us\":[" + std::to_string(h->outer_us[0]) + "," + std::to_string(h->outer_us[1]) + "," + std::to_string(h->outer_us[2]) + "]" + ",\"coarse_unknowns\":" +
                    std::to_string(h->nd) + ",\"device_bytes\":" + std::to_string(h->bytes) + ",\"setup_phase_ms\":{";
    const char* names[8] = {"pattern", "aggregate", "galerkin", "colour", "inverse", "coarse_lu", "vectors",
                            "weights"};
    for (int q = 0; q < 8; ++q) {
        char buf[64];
        snprintf(buf, sizeof buf, "%s\"%s\":%.4f", q ? "," : "", names[q], h->t_phase[q]);
        o += buf;
    }
    o += "},\"tail_level\":" + std::to_string(h->l_tail) + ",\"tail_phases\":" + std::to_string(h->n_tail) +
         ",\"tail_cluster\":" + std::to_string(h->tail_cluster) + ",\"tail_grid\":" + std::to_string(h->tail_grid) +
         ",\"levels\":[";
    for (int l = 0; l < h->nlev; ++l) {
        const Level& L = h->lev[l];
        if (l) o += ",";
        o += "{\"n\":" + std::to_string(L.n) + ",\"nnzb\":" + std::to_string(L.nnzb) +
             ",\"colours\":" + std::to_string(L.n_colours) + ",\"aggregates\":" + std::to_string(L.n_agg) +
             ",\"aggregation_rounds\":" + std::to_string(L.agg_rounds) +
             ",\"colouring_rounds\":" + std::to_string(L.colour_rounds) +
             ",\"smoother_mapping\":\"" + (L.sweep == 2     ? "sweep-split"
                                          : L.sweep        ? "sweep"
                                          : L.bgs_tpr == 7 ? "block-split8"
                                          : L.bgs_tpr == 6 ? "block-split16"
                                          : L.bgs_tpr == 5 ? "wide"
                                          : L.bgs_tpr == 4 ? "staged"
                                          : L.bgs_tpr == 3 ? "thread-split"
                                          : L.bgs_tpr == 2 ? "thread-half"
                                          : L.bgs_tpr      ? "thread"
                                                           : "warp") +
             "\",\"sweep_tiles\":" + std::to_string(L.sw_tiles) + ",\"tune_cached\":" +
             std::to_string(L.tune_cached) + ",\"tune_step_us\":[" +
             std::to_string(L.tune_step_us[0]) + "," + std::to_string(L.tune_step_us[1]) + "," +
             std::to_string(L.tune_step_us[2]) + "]" + ",\"residual_mapping\":\"" +
             (L.spmv_tpr ? "thread" : "warp") + "\",\"tune_us\":[" + std::to_string(L.tune_us[0]) + "," +
             std::to_string(L.tune_us[1]) + "," + std::to_string(L.tune_us[2]) + "," +
             std::to_string(L.tune_us[3]) + "," + std::to_string(L.tune_us[4]) + "," +
             std::to_string(L.tune_us[5]) + "," + std::to_string(L.tune_us[6]) + "," +
             std::to_string(L.tune_us[7]) + "," + std::to_string(L.tune_us[8]) + "," +
             std::to_string(L.tune_us[9]) + "],\"field_major\":" + std::to_string(L.fm) + ",\"smoothed_p\":" + std::to_string(L.smoothed) +
             ",\"p_nnz\":" + std::to_string(L.p_nnz) + ",\"node_damping\":" + (L.omega_s64 ? "1" : "0");
        if (h->nf > 1) {
            o += ",\"field_nodes\":[";
            for (int g = 0; g < h->nf; ++g) o += (g ? "," : "") + std::to_string(L.fo[g + 1] - L.fo[g]);
            o += "]";
        }
        o += "}";
    }
    o += "]}";
    const int len = (int)o.size();
    const int w = len < cap - 1 ? len : cap - 1;
    memcpy(json, o.data(), (size_t)w);
    json[w] = 0;
    return len;
}

// ---------------------------------------------------------------------------
// measurement
// ---------------------------------------------------------------------------
extern "C" int amg_profile(bamg_t h, int enable) {
    if (!h) return BAMG_EINVAL;
    if (enable && !h->prof) {
        // per-colour stored-block counts (all, and those to a lower colour)
        for (int l = 0; l + 1 < h->nlev; ++l) {
            Level& L = h->lev[l];
            std::vector<int> rp((size_t)L.n + 1), ci((size_t)L.nnzb), col((size_t)L.n);
            BAMG_CUDA_TRY(cudaMemcpy(rp.data(), L.rp, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost));
            BAMG_CUDA_TRY(cudaMemcpy(ci.data(), L.ci, sizeof(int) * ci.size(), cudaMemcpyDeviceToHost));
            BAMG_CUDA_TRY(cudaMemcpy(col.data(), L.colour, sizeof(int) * col.size(), cudaMemcpyDeviceToHost));
            L.colour_nnz.assign((size_t)L.n_colours, 0);
            L.colour_nnz_lower.assign((size_t)L.n_colours, 0);
            // (fields on node sets: only blocks of the row's own field are read through x~)
            std::vector<int> fld((size_t)L.n, 0);
            for (int g = 0; h->nf > 1 && g < h->nf; ++g)
                for (int i = L.fo[g]; i < L.fo[g + 1]; ++i) fld[(size_t)i] = g;
            for (int i = 0; i < L.n; ++i) {
                L.colour_nnz[(size_t)col[i]] += rp[i + 1] - rp[i];
                for (int k = rp[i]; k < rp[i + 1]; ++k)
                    if (ci[k] != i && col[ci[k]] < col[i] && fld[(size_t)ci[k]] == fld[(size_t)i])
                        L.colour_nnz_lower[(size_t)col[i]]++;
            }
        }
    }
    h->prof = enable ? 1 : 0;
    if (enable && h->tail_d) TRY(record_tail(h, nullptr, true));
    return BAMG_OK;
}

// resolve every direct-launch record into the per-kind, per-level sums
static int profile_resolve(bamg_ctx* h) {
    for (auto& r : h->recs) {
        BAMG_CUDA_TRY(cudaEventSynchronize(r.e1));
        float e = 0.0f;
        BAMG_CUDA_TRY(cudaEventElapsedTime(&e, r.e0, r.e1));
        if (r.kind >= 0) {
            const int sl = r.level + 1;
            h->acc_ms[r.kind][sl] += e;
            h->acc_bytes[r.kind][sl] += r.bytes;
            h->acc_flops[r.kind][sl] += r.flops;
            h->acc_n[r.kind][sl] += 1;
        }
        h->ev_free.push_back(r.e0);
        h->ev_free.push_back(r.e1);
    }
    h->recs.clear();
    return BAMG_OK;
}

// the sums of kind over level slots s0..s1-1, then cleared
static int profile_take(bamg_ctx* h, int kind, int s0, int s1, double* ms, long long* launches, double* bytes,
                        double* flops) {
    TRY(profile_resolve(h));
    double t = 0.0, by = 0.0, fl = 0.0;
    long long cnt = 0;
    for (int sl = s0; sl < s1; ++sl) {
        t += h->acc_ms[kind][sl];
        by += h->acc_bytes[kind][sl];
        fl += h->acc_flops[kind][sl];
        cnt += h->acc_n[kind][sl];
        h->acc_ms[kind][sl] = h->acc_bytes[kind][sl] = h->acc_flops[kind][sl] = 0.0;
        h->acc_n[kind][sl] = 0;
    }
    if (ms) *ms = t;
    if (launches) *launches = cnt;
    if (bytes) *bytes = by;
    if (flops) *flops = fl;
    return BAMG_OK;
}

extern "C" int amg_profile_read(bamg_t h, int kind, double* ms, long long* launches, double* bytes,
                                double* flops) {
    if (!h || kind < 0 || kind >= BAMG_K_COUNT) return BAMG_EINVAL;
    return profile_take(h, kind, 0, kProfSlots, ms, launches, bytes, flops);
}

extern "C" int amg_profile_read_level(bamg_t h, int kind, int level, double* ms, long long* launches,
                                      double* bytes, double* flops) {
    if (!h || kind < 0 || kind >= BAMG_K_COUNT || level < -1 || level >= h->nlev) return BAMG_EINVAL;
    return profile_take(h, kind, level + 1, level + 2, ms, launches, bytes, flops);
}

// ---------------------------------------------------------------------------
// learned damping
// ---------------------------------------------------------------------------
namespace {
// stream-ordered scratch of one entry point, returned to the pool on exit
struct Scratch {
    cudaStream_t s;
    std::vector<void*> q;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <typename T>
    T* get(size_t count) {
        void* p = nullptr;
        if (pool_alloc(&p, (count ? count : 1) * sizeof(T), s) != cudaSuccess) return nullptr;
        q.push_back(p);
        return static_cast<T*>(p);
    }
    ~Scratch() {
        for (void* p : q) cudaFreeAsync(p, s);
    }
};

int read_flag(int* d_err, cudaStream_t s) {
    int v = 0;
    if (cudaMemcpyAsync(&v, d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return BAMG_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BAMG_ECUDA;
    return map_dev_error(v);
}
}  // namespace

extern "C" int amg_features(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int b,
                            const int* field_of_dof, const int* agg, int n_agg, int level, float* node_feat,
                            float* agg_feat, void* stream) {
    if (!row_ptr || !col_idx || !vals || !field_of_dof || !agg || !node_feat || n_nodes < 1 || n_agg < 1 ||
        n_agg > n_nodes || b < 1 || b > kMaxB || level < 0)
        return BAMG_EINVAL;
    int F = 1;
    if (field_of_dof[0] != 0) return BAMG_EINVAL;
    for (int d = 1; d < b; ++d) {
        const int step = field_of_dof[d] - field_of_dof[d - 1];
        if (step != 0 && step != 1) return BAMG_EINVAL;
        F = field_of_dof[d] + 1;
    }
    if (b % F) return BAMG_EINVAL;
    const int fb = b / F;
    for (int d = 0; d < b; ++d)
        if (field_of_dof[d] != d / fb) return BAMG_EINVAL;
    if (!supported_block(b, fb)) return BAMG_EUNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch w(s);
    int* err = w.get<int>(4);
    int* cnt = w.get<int>((size_t)n_agg + 1);
    if (!err || !cnt) return BAMG_ECUDA;
    BAMG_CUDA_TRY(cudaMemsetAsync(err, 0, 4 * sizeof(int), s));
    TRY(launch_agg_count(n_nodes, n_agg, agg, cnt, err, s));
    TRY(read_flag(err, s));  // aggregate ids in range before they index anything
    TRY(launch_features(b, fb, n_nodes, row_ptr, col_idx, vals, agg, cnt, level, node_feat, err, s));
    if (agg_feat) {
        int* agg_ptr = w.get<int>((size_t)n_agg + 1);
        int* members = w.get<int>((size_t)n_nodes);
        int* tmp = w.get<int>((size_t)n_agg + 1 + scan_tmp_bytes(n_agg) / sizeof(int) + 16);
        if (!agg_ptr || !members || !tmp) return BAMG_ECUDA;
        TRY(build_members(n_nodes, n_agg, agg, agg_ptr, members, tmp, s));
        TRY(launch_agg_features(n_agg, F, agg_ptr, members, node_feat, agg_feat, s));
    }
    return read_flag(err, s);
}

extern "C" int mlp_pack(const float* params, uint16_t* params16, void* stream) {
    if (!params || !params16) return BAMG_EINVAL;
    return launch_pack_half(params, params16, static_cast<cudaStream_t>(stream));
}

extern "C" int mlp_forward(const uint16_t* params16, const float* x, int n, float* y, void* stream) {
    if (n < 0 || (n > 0 && (!params16 || !x || !y))) return BAMG_EINVAL;
    return launch_mlp_forward(params16, x, n, y, static_cast<cudaStream_t>(stream));
}

extern "C" int mlp_grad(const uint16_t* params16, const float* x, const float* t, const int* head, int n, float* grad,
                        float* loss, void* stream) {
    if (n < 1 || !params16 || !x || !t || !head || !grad || !loss) return BAMG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch w(s);
    float* work = w.get<float>(mlp_grad_workspace(n) / sizeof(float) + 1);
    if (!work) return BAMG_ECUDA;
    return launch_mlp_grad(params16, x, t, head, n, grad, loss, work, s);
}

extern "C" int mlp_adam(float* params, uint16_t* params16, const float* grad, float* m, float* v, int t, float lr,
                        float beta1, float beta2, float eps, void* stream) {
    if (t < 1 || !params || !params16 || !grad || !m || !v) return BAMG_EINVAL;
    const float c1 = (float)(1.0 - std::pow((double)beta1, t)), c2 = (float)(1.0 - std::pow((double)beta2, t));
    return launch_adam(params, params16, grad, m, v, lr, beta1, beta2, eps, c1, c2, static_cast<cudaStream_t>(stream));
}

// the captured cycles hold the damping pointers of their kernels: drop them
static void drop_graphs(bamg_ctx* h) {
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->prof_exec) cudaGraphExecDestroy(h->prof_exec);
    if (h->prof_graph) cudaGraphDestroy(h->prof_graph);
    h->graph_exec = nullptr;
    h->graph = nullptr;
    h->prof_exec = nullptr;
    h->prof_graph = nullptr;
    for (auto& r : h->graph_recs) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    h->graph_recs.clear();
}

extern "C" int amg_set_omega(bamg_t h, int level, const double* omega_s, void* stream) {
    if (!h || !omega_s || level < 0 || level >= h->nlev - 1) return BAMG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Level& L = h->lev[level];
    const size_t m = (size_t)L.n * h->F;
    BAMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (!L.omega_s64) {
        // the hierarchy used the scalar damping so far: give this level arrays
        TRY(h->alloc(&L.omega_s64, m));
        if (h->p.cycle_prec == 32) TRY(h->alloc(&L.omega_s32, m));
        BAMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
        drop_graphs(h);
        if (h->tail_d) TRY(record_tail(h, h->stream, false));
    }
    BAMG_CUDA_TRY(cudaMemcpyAsync(L.omega_s64, omega_s, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    if (h->p.cycle_prec == 32) TRY(launch_convert_d2f((long)m, L.omega_s64, L.omega_s32, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    return BAMG_OK;
}

extern "C" int amg_select(bamg_t learned, bamg_t plain, const double* b, double tol, int restart, int max_iter,
                          int* choice, int* iters_learned, int* iters_plain, void* stream) {
    if (!learned || !plain || !b || !choice || learned->nsys != 1 || plain->nsys != 1 || learned->b != plain->b ||
        learned->lev[0].n != plain->lev[0].n)
        return BAMG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t N = (size_t)plain->lev[0].n * plain->b;
    Scratch w(s);
    double* x = w.get<double>(N);
    if (!x) return BAMG_ECUDA;
    int it_l = 0, it_p = 0;
    double rr = 0.0;
    BAMG_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
    const int st_l = fgmres_solve(learned, b, x, tol, restart, max_iter, &it_l, &rr, stream);
    if (st_l < 0) return st_l;
    BAMG_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
    const int st_p = fgmres_solve(plain, b, x, tol, restart, max_iter, &it_p, &rr, stream);
    if (st_p < 0) return st_p;
    // the plain hierarchy judges: the learned one is kept only if it converged in no more iterations
    *choice = (st_l == BAMG_OK && (st_p != BAMG_OK || it_l <= it_p)) ? 0 : 1;
    if (iters_learned) *iters_learned = it_l;
    if (iters_plain) *iters_plain = it_p;
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    return BAMG_OK;
}

extern "C" int amg_level_omega(bamg_t h, int level, double* omega_s, double* omega_p) {
    if (!h || level < 0 || level >= h->nlev - 1) return BAMG_EINVAL;
    const Level& L = h->lev[level];
    BAMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (omega_s) {
        const size_t m = (size_t)L.n * h->F;
        if (L.omega_s64) BAMG_CUDA_TRY(cudaMemcpy(omega_s, L.omega_s64, sizeof(double) * m, cudaMemcpyDeviceToHost));
        else
            for (size_t e = 0; e < m; ++e) omega_s[e] = h->p.omega;
    }
    if (omega_p) {
        const size_t m = (size_t)L.n_agg * h->F;
        if (L.omega_p64 && L.smoothed)
            BAMG_CUDA_TRY(cudaMemcpy(omega_p, L.omega_p64, sizeof(double) * m, cudaMemcpyDeviceToHost));
        else
            for (size_t e = 0; e < m; ++e) omega_p[e] = 0.0;
    }
    return BAMG_OK;
}

extern "C" int amg_level_p(bamg_t h, int level, int* nnz, int* p_rp, int* p_ci, double* p_v) {
    if (!h || !nnz || level < 0 || level >= h->nlev - 1) return BAMG_EINVAL;
    const Level& L = h->lev[level];
    *nnz = L.smoothed ? L.p_nnz : 0;
    if (!L.smoothed) return BAMG_OK;
    BAMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (p_rp) BAMG_CUDA_TRY(cudaMemcpy(p_rp, L.p_rp, sizeof(int) * (size_t)(L.n + 1), cudaMemcpyDeviceToHost));
    if (p_ci) BAMG_CUDA_TRY(cudaMemcpy(p_ci, L.p_ci, sizeof(int) * (size_t)L.p_nnz, cudaMemcpyDeviceToHost));
    if (p_v)
        BAMG_CUDA_TRY(cudaMemcpy(p_v, L.p_v64, sizeof(double) * (size_t)L.p_nnz * h->F * h->fb * h->fb,
                                 cudaMemcpyDeviceToHost));
    return BAMG_OK;
}
