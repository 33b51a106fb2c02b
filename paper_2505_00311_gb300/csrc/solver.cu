// solver.cu -- host side of the PDCS library: pdcs_create (validation, row
// grouping by cone kind, K' build, diagonal rescaling on the device), the
// iteration schedule (one CUDA graph per check period) and the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/pdcs.h"
#include "common.cuh"
#include "cone_math.cuh"
#include "dev.h"
#include "launch.h"
#include "setup_kernels.cuh"
#include "state.h"

using namespace pdcs;

namespace {

std::string g_create_error;  // text of the last failed pdcs_create
std::string g_batch_error;   // text of the last failed pdcs_batch_create

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int pow2_floor(int v) {
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

// Device memory arena: one cudaMalloc, buffers carved at 256-byte boundaries.
struct Arena {
    char* base = nullptr;
    size_t cap = 0, used = 0;
    size_t plan = 0;
    template <typename T>
    void reserve(size_t count) { plan += ((count * sizeof(T) + 255) / 256) * 256; }
    template <typename T>
    T* take(size_t count) {
        size_t bytes = ((count * sizeof(T) + 255) / 256) * 256;
        T* p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return p;
    }
};

// SpMV plan of one matrix: rows binned by length (see spmv_binned), the matrix
// stored bin by bin, and the unroll.
// Or (sliced) the matrix in slices of 32 rows of similar length (see spmv_sliced).
enum { kFormatBinned = 1, kFormatSliced = 2 };
struct SpmvPlan {
    int format = kFormatBinned;
    SpmvBins B{};
    int* list = nullptr;  // device row list, bin by bin: binned row i is row list[i]
    int* rp = nullptr;    // device row pointer over the binned rows
    int* ci = nullptr;    // device columns, bin by bin (sliced: in the sliced storage)
    int shift = 3;        // lanes = 2^(ceil(log2(length)) - shift), clamped to 1..32
    int unroll = 4;
    SlicePlan S{};        // sliced format: the plan (device arrays below)
};

// Host side of a sliced plan: rows of at most kSliceMaxLen entries sorted by length
// (longest first, then by row), cut into slices whose lanes per row S follow from the
// slice's first (longest) row; longer rows after them in row order.
struct SliceHost {
    std::vector<int> slice_off, out_row, long_row, long_rp;
    std::vector<unsigned char> slice_lg;
    long long entries = 0;  // sliced storage size (padding included)
};

void plan_slices(const std::vector<int>& rp, int rows, SliceHost& H) {
    std::vector<int> cnt(kSliceMaxLen + 2, 0), shorts;
    H.long_row.clear();
    for (int r = 0; r < rows; ++r) {
        const int len = rp[r + 1] - rp[r];
        if (len > kSliceMaxLen) H.long_row.push_back(r);
        else ++cnt[len];
    }
    // counting sort by decreasing length, stable in the row index
    std::vector<int> start(kSliceMaxLen + 2, 0);
    int acc = 0;
    for (int len = kSliceMaxLen; len >= 0; --len) { start[len] = acc; acc += cnt[len]; }
    shorts.assign(acc, 0);
    for (int r = 0; r < rows; ++r) {
        const int len = rp[r + 1] - rp[r];
        if (len <= kSliceMaxLen) shorts[start[len]++] = r;
    }
    H.slice_off.clear();
    H.slice_lg.clear();
    H.out_row.clear();
    long long off = 0;
    for (int i = 0; i < acc;) {
        const int L = rp[shorts[i] + 1] - rp[shorts[i]];
        int lg = 0;
        while (lg < 5 && L > (2 << lg) * kSlicePairsPerLane) ++lg;
        const int S = 1 << lg, h = 32 >> lg;
        const int W = (L + 2 * S - 1) / (2 * S) * (2 * S);  // width: a multiple of 2 S
        H.slice_off.push_back((int)off);
        H.slice_lg.push_back((unsigned char)lg);
        for (int j = 0; j < 32; ++j) H.out_row.push_back(j < h && i + j < acc ? shorts[i + j] : -1);
        off += 32LL * W / S;  // h rows of W entries
        i += h;
    }
    H.slice_off.push_back((int)off);
    H.long_rp.assign(H.long_row.size() + 1, 0);
    for (size_t j = 0; j < H.long_row.size(); ++j) {
        H.long_rp[j] = (int)off;
        off += rp[H.long_row[j] + 1] - rp[H.long_row[j]];
    }
    H.long_rp[H.long_row.size()] = (int)off;
    H.entries = off;
}

}  // namespace

struct pdcs_ctx {
    pdcs_options opt;
    int m = 0, n = 0;
    long long nnz = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int sms = 152;

    // row grouping: internal row r holds original row perm[r]
    std::vector<int> perm;
    int m_zero = 0, m_scalar = 0, n_soc = 0, exp_row0 = 0, n_exp = 0;

    Arena arena;
    // device buffers (FP64 path)
    int *rp = nullptr, *ci = nullptr, *rpT = nullptr, *ciT = nullptr;
    double *val0 = nullptr, *val0T = nullptr, *val = nullptr, *valT = nullptr;
    double *valb = nullptr, *valbT = nullptr;  // K~, K~' bin by bin (in the memory of val0, val0T)
    double *c0 = nullptr, *h0 = nullptr, *l0 = nullptr, *u0 = nullptr;
    double *cs = nullptr, *hs = nullptr, *ls = nullptr, *us = nullptr;
    double *dr = nullptr, *dc = nullptr, *rn = nullptr, *cn = nullptr;
    int *soc_off = nullptr, *soc_dim = nullptr;
    unsigned char* soc_rot = nullptr;
    int *tie_off = nullptr, *tie_len = nullptr;
    int n_tie = 0;
    float *soc_lam = nullptr, *exp_L = nullptr;
    double *soc_w = nullptr, *soc_wp = nullptr, *exp_lg = nullptr;
    double* part = nullptr;
    Ctrl* ctrl = nullptr;
    double* scal = nullptr;  // small scalar scratch
    Ctrl* h_ctrl = nullptr;  // pinned host mirror

    Dev<double> D;
    std::vector<pdcs_cone> pcones;  // primal cone blocks (options.primal_cones, copied)
    long long pc_start = 0;
    SpmvPlan pk, pkt;  // K (m rows) and K' (n rows)
    // FP32-iterate mode: FP32 copies of K~, K~', c~, h~, l~, u~ and the iterate state;
    // checks, restarts and the final phase stay FP64 (D)
    Dev<float> DF;
    float *val_f = nullptr, *valT_f = nullptr;  // in the SpMV storage
    bool fp32_active = false;          // the FP32 phase is running
    double fp32_best = INFINITY;       // best relative KKT error seen in the FP32 phase
    int fp32_stall = 0;                // checks since it last improved by 10 %
    int g_vec_n = 0, g_vec_m = 0, g_dual = 0, g_kktd = 0;

    cudaGraphExec_t graph = nullptr, graph32 = nullptr;
    cudaStream_t aux[2] = {nullptr, nullptr};  // helper streams of the concurrent dual-update roles
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
    int launches_per_attempt = 4;
    int team_cones = 0;  // SOC cones projected grid-wise
    bool fuse_primal = false;  // the K' product forms the next primal update (spmv_kt_primal)
    bool started = false;
    double setup_seconds = 0.0, solve_seconds = 0.0;
    double norm2 = 0.0;
    long long launches = 0;
    int last_status = PDCS_OK;

    ~pdcs_ctx() {
        for (int k = 0; k < 2; ++k) {
            if (aux[k]) cudaStreamDestroy(aux[k]);
            if (ev_join[k]) cudaEventDestroy(ev_join[k]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (graph) cudaGraphExecDestroy(graph);
        if (graph32) cudaGraphExecDestroy(graph32);
        if (arena.base) cudaFree(arena.base);
        if (h_ctrl) cudaFreeHost(h_ctrl);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return e_ == cudaErrorMemoryAllocation ? PDCS_ERR_OOM : PDCS_ERR_CUDA;        \
        }                                                                                 \
    } while (0)

namespace {

template <typename T>
void launch_spmv(const SpmvPlan& P, cudaStream_t s, const int* rp, const int* ci, const T* val, const T* x, T* y0,
                 T* y1, const Ctrl* ctrl, int sel, int skip, const T* xalt = nullptr) {
    if (P.format == kFormatSliced) k_spmv_sliced(P.S, s, ci, val, x, y0, y1, ctrl, sel, skip, xalt);
    else k_spmv(P.B, P.unroll, s, P.list, rp, ci, val, x, y0, y1, ctrl, sel, skip);
}

// Bins of a CSR matrix: lanes per row 2^(ceil(log2(len)) - shift) clamped to 1..32 (or
// `fixed` for every row), bins ordered by decreasing lanes, rows increasing within a
// bin; a bin gets enough blocks for one pass over its rows (at most 32 per SM).
void plan_bins(const std::vector<int>& rp, int rows, int shift, int fixed, int sms, std::vector<int>& list,
               SpmvBins& B) {
    std::vector<unsigned char> bin_of(rows);
    long long cnt[kSpmvMaxBins] = {0};
    for (int r = 0; r < rows; ++r) {
        int lanes = fixed;
        if (lanes <= 0) {
            const int len = rp[r + 1] - rp[r];
            int lg = 0;
            while ((1 << lg) < len) ++lg;  // ceil(log2(len))
            lanes = 1 << std::min(5, std::max(0, lg - shift));
        }
        int k = 0;  // bin 0: 32 lanes ... bin 5: 1 lane
        while ((32 >> k) > lanes) ++k;
        bin_of[r] = (unsigned char)k;
        ++cnt[k];
    }
    list.resize(rows);
    long long pos[kSpmvMaxBins] = {0};
    B.nbins = 0;
    int blk = 0, row = 0;
    for (int k = 0; k < kSpmvMaxBins; ++k) {
        if (!cnt[k]) continue;
        const int lanes = 32 >> k;
        const long long rows_per_block = (long long)kWarpsPerBlock * (32 / lanes);
        const long long nb = std::min((cnt[k] + rows_per_block - 1) / rows_per_block, (long long)sms * 32);
        B.blk[B.nbins] = blk;
        B.row[B.nbins] = row;
        B.lanes[B.nbins] = lanes;
        pos[k] = row;
        blk += (int)nb;
        row += (int)cnt[k];
        ++B.nbins;
    }
    B.blk[B.nbins] = blk;
    B.row[B.nbins] = row;
    for (int r = 0; r < rows; ++r) list[pos[bin_of[r]]++] = r;
}

// Process-wide cache of tuned SpMV plans (shift, unroll), keyed by matrix signature.
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;

std::string spmv_signature(const std::vector<int>& rp, int rows) {
    long long hist[40] = {0};
    for (int r = 0; r < rows; ++r) {
        const int len = rp[r + 1] - rp[r];
        int lg = 0;
        while ((1 << lg) < len && lg < 39) ++lg;
        ++hist[lg];
    }
    std::string sig = std::to_string(rows) + ":" + std::to_string(rp[rows]);
    for (int k = 0; k < 40; ++k)
        if (hist[k]) sig += ":" + std::to_string(k) + "=" + std::to_string(hist[k]);
    return sig;
}

int spmv_grid(int rows, int G, int sms) {
    long long rows_per_block = (long long)kWarpsPerBlock * (32 / G);
    long long g = (rows + rows_per_block - 1) / rows_per_block;
    return (int)std::max(1LL, std::min(g, (long long)sms * 32));
}

int vec_grid(long long k, int sms, int per_sm = 8) {
    long long g = (k + kBlock - 1) / kBlock;
    return (int)std::max(1LL, std::min(g, (long long)sms * per_sm));
}


// Kernel classes of pdcs_kernel_times (see include/pdcs.h).
constexpr int kKernelClasses = 12;

// Optional CUDA-event recorder for kernel timing: event pairs per kernel class.
struct Prof {
    std::vector<cudaEvent_t> ev[kKernelClasses];
    void mark(int cls, cudaStream_t s) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) == cudaSuccess) {
            cudaEventRecord(e, s);
            ev[cls].push_back(e);
        }
    }
};

// Binned row pointer of a row list (host).
void binned_rowptr(const std::vector<int>& rp, const std::vector<int>& list, std::vector<int>& rpb) {
    rpb.resize(list.size() + 1);
    rpb[0] = 0;
    for (size_t i = 0; i < list.size(); ++i) rpb[i + 1] = rpb[i] + (rp[list[i] + 1] - rp[list[i]]);
}

// Stores a matrix (rows in order: host rp, device drp, dci, dval) bin by bin for the
// row list `list` of plan P: uploads the list and the binned row pointer into P.list,
// P.rp and gathers the values (as TD) into valb and, when cols, the columns into P.ci.
template <typename TD>
cudaError_t store_binned(pdcs_ctx* ctx, SpmvPlan& P, const std::vector<int>& rp, const std::vector<int>& list,
                         const int* drp, const int* dci, const double* dval, TD* valb, bool cols) {
    const int rows = (int)list.size();
    if (rows <= 0) return cudaSuccess;
    std::vector<int> rpb;
    binned_rowptr(rp, list, rpb);
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(P.list, list.data(), sizeof(int) * rows, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.rp, rpb.data(), sizeof(int) * (rows + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const long long g = std::min(((long long)rows + kWarpsPerBlock - 1) / kWarpsPerBlock, (long long)ctx->sms * 32);
        k_bin_rows_copy((int)g, s, rows, P.list, drp, dci, dval, P.rp, cols ? P.ci : nullptr, valb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors are pageable
    return e;
}

// Uploads the sliced plan H of P (arrays taken from the arena beforehand) and fills the
// sliced storage of a matrix (rows in order: device drp, dci, dval) with values as TD
// (cols: also the columns into P.ci).
template <typename TD>
cudaError_t store_sliced(pdcs_ctx* ctx, SpmvPlan& P, const SliceHost& H, const int* drp, const int* dci,
                         const double* dval, TD* vals, bool cols) {
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaSuccess;
    if (cols) {
        unsigned char* slg = const_cast<unsigned char*>(P.S.slice_lg);
        if (!H.slice_lg.empty())
            e = cudaMemcpyAsync(slg, H.slice_lg.data(), H.slice_lg.size(), cudaMemcpyHostToDevice, s);
        int* so = const_cast<int*>(P.S.slice_off);
        int* orow = const_cast<int*>(P.S.out_row);
        int* lr = const_cast<int*>(P.S.long_row);
        int* lrp = const_cast<int*>(P.S.long_rp);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(so, H.slice_off.data(), sizeof(int) * H.slice_off.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !H.out_row.empty())
            e = cudaMemcpyAsync(orow, H.out_row.data(), sizeof(int) * H.out_row.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !H.long_row.empty())
            e = cudaMemcpyAsync(lr, H.long_row.data(), sizeof(int) * H.long_row.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(lrp, H.long_rp.data(), sizeof(int) * H.long_rp.size(), cudaMemcpyHostToDevice, s);
    }
    const long long slots = 32LL * P.S.nslices + P.S.nlong;
    if (e == cudaSuccess && slots > 0) {
        const int g = (int)std::max(1LL, std::min((slots + kBlock - 1) / kBlock, (long long)ctx->sms * 16));
        k_sliced_copy(P.S, g, s, drp, dci, dval, cols ? P.ci : nullptr, vals);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors are pageable
    return e;
}

// Times the candidate plans of one matrix (bin shift 1..4, unroll 1, 2, 4; 3 warm-up and
// 20 timed launches each on the given vectors, in the value type T the iterations use,
// each on the matrix stored for its bins) and keeps the fastest in P, with the matrix
// stored bin by bin for it (columns in P.ci, values as T in valb).  The choice is cached
// per process by the matrix signature and T.
template <typename T>
cudaError_t tune_spmv(pdcs_ctx* ctx, SpmvPlan& P, const std::vector<int>& rp, int rows, const int* drp,
                      const int* dci, const double* dval, T* valb, const T* x, T* y) {
    cudaStream_t s = ctx->stream;
    if (rows <= 0) return cudaSuccess;
    const std::string sig = spmv_signature(rp, rows) + (sizeof(T) == 4 ? ":f32" : ":f64");
    int shift = P.shift, unroll = P.unroll;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(sig);
        if (it != g_tune_cache.end()) { shift = it->second.first; unroll = it->second.second; cached = true; }
    }
    std::vector<int> list;
    cudaError_t e = cudaSuccess;
    if (!cached) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
        if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
        float best = 1e30f;
        for (int sh = 1; sh <= 4 && e == cudaSuccess; ++sh) {
            SpmvPlan c = P;
            plan_bins(rp, rows, sh, 0, ctx->sms, list, c.B);
            e = store_binned<T>(ctx, P, rp, list, drp, dci, dval, valb, true);
            for (int un = 1; un <= 4 && e == cudaSuccess; un *= 2) {
                c.shift = sh;
                c.unroll = un;
                for (int r = 0; r < 3; ++r) launch_spmv<T>(c, s, P.rp, P.ci, valb, x, y, nullptr, nullptr, 0, 0);
                cudaEventRecord(e0, s);
                for (int r = 0; r < 20; ++r) launch_spmv<T>(c, s, P.rp, P.ci, valb, x, y, nullptr, nullptr, 0, 0);
                cudaEventRecord(e1, s);
                e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaGetLastError();
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e == cudaSuccess && ms < best) { best = ms; shift = sh; unroll = un; }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[sig] = std::make_pair(shift, unroll);
    }
    P.shift = shift;
    P.unroll = unroll;
    plan_bins(rp, rows, shift, 0, ctx->sms, list, P.B);
    return store_binned<T>(ctx, P, rp, list, drp, dci, dval, valb, true);
}

constexpr int kLaunchesPerAttempt = 4;  // batches: one dual-update launch per evaluation
constexpr int kLaunchesPerCheck = 12;

// the dual update: its three cone roles as concurrent kernels (forked from the context's
// stream onto two helper streams and joined back; captured as parallel graph branches),
// or one launch over all roles for a program set up to join a batch (its grid includes
// idle blocks that take part in the step controller's block count)
template <typename T>
void enqueue_dual(pdcs_ctx* ctx, const Dev<T>& DT) {
    cudaStream_t s = ctx->stream;
    if (ctx->opt.batch_blocks > 0) {
        k_dual_update(DT, ctx->g_dual, s);
        return;
    }
    const bool team = DT.team_nb > 0;  // the grid-wise cones follow the SOC role on its stream
    const int roles = (DT.nb_scal > 0) + (DT.nb_soc > 0 || team) + (DT.nb_exp > 0);
    if (roles <= 1) {
        k_dual_exp(DT, s);
        k_dual_soc(DT, s);
        if (team) k_soc_team(DT, 0, s);
        k_dual_scalar(DT, s);
        return;
    }
    cudaEventRecord(ctx->ev_fork, s);
    cudaStreamWaitEvent(ctx->aux[0], ctx->ev_fork, 0);
    cudaStreamWaitEvent(ctx->aux[1], ctx->ev_fork, 0);
    k_dual_soc(DT, ctx->aux[0]);
    if (team) k_soc_team(DT, 0, ctx->aux[0]);
    k_dual_scalar(DT, ctx->aux[1]);
    k_dual_exp(DT, s);
    cudaEventRecord(ctx->ev_join[0], ctx->aux[0]);
    cudaEventRecord(ctx->ev_join[1], ctx->aux[1]);
    cudaStreamWaitEvent(s, ctx->ev_join[0], 0);
    cudaStreamWaitEvent(s, ctx->ev_join[1], 0);
}

// one PDHG evaluation on the state DT (FP64, or FP32 in the FP32 phase) with the matrix
// copies of its precision
template <typename T>
void enqueue_attempt_t(pdcs_ctx* ctx, Dev<T>& DT, Prof* P) {
    cudaStream_t s = ctx->stream;
    if (P) P->mark(0, s);
    k_primal_update(DT, ctx->g_vec_n, s);
    k_pc(DT, kPcHat, 1, s);  // primal cone blocks of x-hat
    if (P) { P->mark(0, s); P->mark(1, s); }
    launch_spmv<T>(ctx->pk, s, DT.rp, DT.ci, DT.val, DT.xh, DT.kxh0, DT.kxh1, DT.ctrl, 1, 1, DT.xh1);
    if (P) { P->mark(1, s); P->mark(2, s); }
    enqueue_dual(ctx, DT);
    if (P) { P->mark(2, s); P->mark(3, s); }
    if (ctx->fuse_primal) k_spmv_kt_primal(ctx->pkt.S, s, DT.ciT, DT.valT, DT);  // + next primal update
    else launch_spmv<T>(ctx->pkt, s, DT.rpT, DT.ciT, DT.valT, DT.yh, DT.ktyh, nullptr, DT.ctrl, 0, 2);
    if (P) P->mark(3, s);
    ctx->launches += ctx->launches_per_attempt;
}

// restart / termination check (or the initial evaluation of the anchor): candidates
// from the state DT, their products and KKT always in FP64
template <typename T>
void enqueue_check_t(pdcs_ctx* ctx, Dev<T>& DT, Prof* P) {
    cudaStream_t s = ctx->stream;
    Dev<double>& D = ctx->D;
    auto mark = [&](int c) { if (P) P->mark(c, s); };
    mark(4);
    ctx->launches += kLaunchesPerCheck + (DT.team_nb > 0 ? 2 : 0) + (DT.n_pc > 0 ? 4 : 0);
    mark(5);
    k_flush_primal(DT, ctx->g_vec_n, s);
    k_flush_dual(DT, ctx->g_vec_m, s);
    mark(5); mark(6);
    k_cand_primal(DT, dim3(ctx->g_vec_n, 2), s);
    k_pc(DT, kPcCand, 2, s);
    mark(6); mark(7);
    k_cand_dual(DT, dim3(ctx->g_dual, 2), s);
    k_soc_team(DT, 1, s);
    mark(7); mark(8);
    for (int q = 0; q < 2; ++q) {
        launch_spmv<double>(ctx->pk, s, D.rp, D.ci, D.val, D.xc + (size_t)q * ctx->n,
                                    D.kxc + (size_t)q * ctx->m, nullptr, D.ctrl, 0, 1);
        launch_spmv<double>(ctx->pkt, s, D.rpT, D.ciT, D.valT,
                                    D.yc + (size_t)q * ctx->m, D.ktyc + (size_t)q * ctx->n, nullptr, D.ctrl, 0, 1);
    }
    mark(8); mark(9);
    k_kkt_primal(DT, dim3(ctx->g_dual, 2), s);
    k_soc_team(DT, 2, s);
    mark(9); mark(10);
    k_pc(DT, kPcLam, 2, s);  // the candidates' reduced costs on the primal cone blocks
    k_kkt_dual(DT, ctx->g_kktd, s);
    mark(10); mark(11);
    k_restart_primal(DT, ctx->g_vec_n, s);
    k_restart_dual(DT, ctx->g_vec_m, s);
    mark(11);
    mark(4);
}

void enqueue_attempt(pdcs_ctx* ctx, Prof* P = nullptr) {
    if (ctx->fp32_active) enqueue_attempt_t<float>(ctx, ctx->DF, P);
    else enqueue_attempt_t<double>(ctx, ctx->D, P);
}

void enqueue_check(pdcs_ctx* ctx, Prof* P = nullptr) {
    if (ctx->fp32_active) enqueue_check_t<float>(ctx, ctx->DF, P);
    else enqueue_check_t<double>(ctx, ctx->D, P);
}

// After a flush: no pending update, no precomputed x-hat, and x-hat in the first buffer
// (xhat_first copies it there first).
__global__ void clear_pending(Ctrl* C) {
    C->pending = 0;
    C->xnext = 0;
    C->xsel = 0;
}

template <typename T>
__global__ void xhat_first(int n, T* xh, const T* __restrict__ xh1, const Ctrl* C) {
    if (!C->xsel) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) xh[j] = xh1[j];
}

__global__ void widen(int k, const float* __restrict__ in, double* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) out[i] = (double)in[i];
}

pdcs_status read_ctrl(pdcs_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->h_ctrl, ctx->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PDCS_OK;
}

bool finite_all(const double* a, long long k) {
    if (!a) return true;
    for (long long i = 0; i < k; ++i)
        if (std::isnan(a[i])) return false;
    return true;
}

pdcs_status build(pdcs_ctx* ctx, const pdcs_csr* K, const double* c, const double* h, const double* lb,
                  const double* ub, const pdcs_cone* cones, int64_t n_cones) {
    const int m = ctx->m, n = ctx->n;
    const long long nnz = ctx->nnz;
    // ---- row grouping: zero rows, nonnegative rows, SOC/RSOC blocks, exp cones
    std::vector<int> zero_rows, nonneg_rows, soc_o, soc_d, exp_o;
    std::vector<unsigned char> soc_r, exp_k;  // exp_k: 1 for a K_exp^* (EXP_DUAL) block
    {
        long long o = 0;
        for (int64_t k = 0; k < n_cones; ++k) {
            const int t = cones[k].type;
            const long long d = cones[k].dim;
            if (t == PDCS_CONE_ZERO) for (long long i = 0; i < d; ++i) zero_rows.push_back((int)(o + i));
            else if (t == PDCS_CONE_NONNEG) for (long long i = 0; i < d; ++i) nonneg_rows.push_back((int)(o + i));
            else if (t == PDCS_CONE_SOC || t == PDCS_CONE_RSOC) {
                soc_o.push_back((int)o); soc_d.push_back((int)d); soc_r.push_back(t == PDCS_CONE_RSOC);
            } else {
                exp_o.push_back((int)o);
                exp_k.push_back(t == PDCS_CONE_EXP_DUAL);
            }
            o += d;
        }
    }
    ctx->perm.clear();
    ctx->perm.reserve(m);
    for (int r : zero_rows) ctx->perm.push_back(r);
    for (int r : nonneg_rows) ctx->perm.push_back(r);
    ctx->m_zero = (int)zero_rows.size();
    ctx->m_scalar = (int)(zero_rows.size() + nonneg_rows.size());
    std::vector<int> soc_off_i(soc_o.size());
    for (size_t k = 0; k < soc_o.size(); ++k) {
        soc_off_i[k] = (int)ctx->perm.size();
        for (int i = 0; i < soc_d[k]; ++i) ctx->perm.push_back(soc_o[k] + i);
    }
    ctx->exp_row0 = (int)ctx->perm.size();
    for (int o : exp_o) for (int i = 0; i < 3; ++i) ctx->perm.push_back(o + i);
    ctx->n_soc = (int)soc_o.size();
    ctx->n_exp = (int)exp_o.size();
    // tie groups for the rescaling: RSOC first two rows (per coordinate), whole blocks (block mode)
    std::vector<int> tie_o, tie_l;
    if (ctx->opt.rescale != PDCS_RESCALE_NONE) {
        for (int k = 0; k < ctx->n_soc; ++k) {
            if (ctx->opt.rescale == PDCS_RESCALE_BLOCK) { tie_o.push_back(soc_off_i[k]); tie_l.push_back(soc_d[k]); }
            else if (soc_r[k]) { tie_o.push_back(soc_off_i[k]); tie_l.push_back(2); }
        }
        if (ctx->opt.rescale == PDCS_RESCALE_BLOCK)
            for (int e = 0; e < ctx->n_exp; ++e) { tie_o.push_back(ctx->exp_row0 + 3 * e); tie_l.push_back(3); }
    }
    ctx->n_tie = (int)tie_o.size();
    // primal cone blocks: first variable, size and rotation of each, chunks of the largest
    const int n_pc = (int)ctx->pcones.size();
    std::vector<int> pc_o(n_pc + 1, 0), pc_dd(n_pc + 1, 0);
    std::vector<unsigned char> pc_r(n_pc + 1, 0);
    int pc_len = 0, pc_nch = 1;
    for (int k = 0; k < n_pc; ++k) {
        pc_o[k] = (int)ctx->pc_start + pc_len;
        pc_dd[k] = (int)ctx->pcones[k].dim;
        pc_r[k] = ctx->pcones[k].type == PDCS_CONE_RSOC;
        pc_len += pc_dd[k];
        pc_nch = std::max(pc_nch, (pc_dd[k] + kPcChunk - 1) / kPcChunk);
    }
    if (n_pc > 0 && (long long)n_pc * pc_nch > (1LL << 24)) {
        ctx->err = "too many primal cone blocks for one launch";
        return PDCS_ERR_INVALID;
    }

    // ---- internal K (rows permuted) and K' by counting sort (host, once)
    std::vector<int> rp_i(m + 1), ci_i((size_t)nnz);
    std::vector<double> v_i((size_t)nnz);
    rp_i[0] = 0;
    for (int r = 0; r < m; ++r) {
        const int src = ctx->perm[r];
        const long long b = K->row_ptr[src], e = K->row_ptr[src + 1];
        const int dst = rp_i[r];
        for (long long p = b; p < e; ++p) {
            ci_i[dst + (p - b)] = K->col[p];
            v_i[dst + (p - b)] = K->val[p];
        }
        rp_i[r + 1] = dst + (int)(e - b);
    }
    std::vector<int> rpT(n + 1, 0), ciT((size_t)nnz);
    std::vector<double> vT((size_t)nnz);
    for (long long p = 0; p < nnz; ++p) rpT[ci_i[p] + 1]++;
    for (int j = 0; j < n; ++j) rpT[j + 1] += rpT[j];
    {
        std::vector<int> cur(rpT.begin(), rpT.end() - 1);
        for (int r = 0; r < m; ++r)
            for (int p = rp_i[r]; p < rp_i[r + 1]; ++p) {
                const int q = cur[ci_i[p]]++;
                ciT[q] = r;
                vT[q] = v_i[p];
            }
    }
    // ---- SpMV storage: sliced (single programs) or binned (batches, fixed lane counts)
    int fmt = ctx->opt.spmv_format;
    if (fmt == 0) fmt = (ctx->opt.batch_blocks > 0 || ctx->opt.spmv_lanes != 0) ? kFormatBinned : kFormatSliced;
    SliceHost hk, hkt;
    if (fmt == kFormatSliced) {
        plan_slices(rp_i, m, hk);
        plan_slices(rpT, n, hkt);
        if (hk.entries >= 0x7fffffffLL || hkt.entries >= 0x7fffffffLL) fmt = kFormatBinned;
    }
    const bool sliced = fmt == kFormatSliced;
    ctx->pk.format = ctx->pkt.format = fmt;
    const long long eK = sliced ? std::max(nnz, hk.entries) : nnz;    // storage entries of K~
    const long long eKT = sliced ? std::max(nnz, hkt.entries) : nnz;  // and of K~'
    std::vector<double> h_i(m), l_h(n), u_h(n);
    for (int r = 0; r < m; ++r) h_i[r] = h[ctx->perm[r]];
    for (int j = 0; j < n; ++j) {
        l_h[j] = lb ? lb[j] : 0.0;
        u_h[j] = ub ? ub[j] : INFINITY;
    }
    double hmax = 0.0, cmax = 0.0;
    for (int i = 0; i < m; ++i) hmax = std::max(hmax, std::fabs(h[i]));
    for (int j = 0; j < n; ++j) cmax = std::max(cmax, std::fabs(c[j]));

    // ---- device memory plan
    std::vector<int> list_k, list_kt;  // SpMV row lists (default plans; tuned below on request)
    plan_bins(rp_i, m, ctx->pk.shift, ctx->opt.spmv_lanes, ctx->sms, list_k, ctx->pk.B);
    plan_bins(rpT, n, ctx->pkt.shift, ctx->opt.spmv_lanes, ctx->sms, list_kt, ctx->pkt.B);
    ctx->g_vec_n = vec_grid(n, ctx->sms);
    ctx->g_vec_m = vec_grid(m, ctx->sms);
    ctx->g_kktd = vec_grid(n, ctx->sms);
    int nb_scal = ctx->m_scalar > 0 ? vec_grid(ctx->m_scalar, ctx->sms) : 0;
    int nb_soc = ctx->n_soc > 0 ? (int)std::min<long long>((ctx->n_soc + kWarpsPerBlock - 1) / kWarpsPerBlock,
                                                           (long long)ctx->sms * 8)
                                : 0;
    // SOC tiles of the FP64 dual update (soc_lane_entries = E > 0): cones sorted by dimension
    // (largest first); a tile is up to 32 / S cones sharing the lane-group size S of its first
    // cone, S the smallest power of two with dim <= S E and (32 / S) dim <= kSocTileRows;
    // cones longer than kSocTileRows rows (all cones when E = 0) come last, a warp each
    std::vector<int> t_cone0, t_row0, t_order, t_trow, t_so;
    std::vector<unsigned char> t_lg;
    int n_large = 0;
    // grid-wise cones (team.cuh): by default those of at least kTeamMinDim rows that alone
    // hold more than one SM's share of the SOC rows, whose FP64 work a warp (or a block)
    // would otherwise serialise on one SM; soc_grid_dim > 0 takes every cone of at least
    // that many rows, -1 none.  Single programs with FP64 iterates only.
    std::vector<unsigned char> huge(ctx->n_soc + 1, 0);
    std::vector<int> team_cone, team_b0, team_g;
    int team_nb = 0;
    if (ctx->opt.batch_blocks == 0 && ctx->n_soc > 0 && ctx->opt.soc_grid_dim >= 0 &&
        ctx->opt.precision == PDCS_PRECISION_FP64) {
        long long soc_rows = 0;
        for (int k = 0; k < ctx->n_soc; ++k) soc_rows += soc_d[k];
        std::vector<int> hc;
        for (int k = 0; k < ctx->n_soc; ++k) {
            const long long dk = soc_d[k];
            const bool h = ctx->opt.soc_grid_dim > 0 ? dk >= ctx->opt.soc_grid_dim
                                                     : (dk >= kTeamMinDim && dk * ctx->sms > soc_rows);
            if (h) hc.push_back(k);
        }
        int occ = 0;
        if (!hc.empty()) occ = k_team_occupancy((const Dev<double>*)nullptr);
        if (!hc.empty() && occ >= 1) {
            team_nb = ctx->sms;
            std::stable_sort(hc.begin(), hc.end(), [&](int a, int b) { return soc_d[a] > soc_d[b]; });
            const int nh = (int)hc.size();
            if (nh > team_nb) {  // one block per cone, dealt round-robin (largest first)
                for (int i = 0; i < nh; ++i) {
                    team_cone.push_back(hc[i]); team_b0.push_back(i % team_nb); team_g.push_back(1);
                }
            } else {  // one block each, the rest shared in proportion to the rows
                long long tot = 0;
                for (int c : hc) tot += soc_d[c];
                int b0 = 0;
                for (int c : hc) {
                    long long g = 1 + (long long)(team_nb - nh) * soc_d[c] / tot;
                    g = std::min<long long>(g, std::max<long long>(1, (soc_d[c] - 1 + kTeamMinRows - 1) / kTeamMinRows));
                    team_cone.push_back(c); team_b0.push_back(b0); team_g.push_back((int)g);
                    b0 += (int)g;
                }
            }
            for (int c : hc) huge[c] = 1;
        }
    }
    {
        std::vector<int> ord(ctx->n_soc);
        for (int k = 0; k < ctx->n_soc; ++k) ord[k] = k;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return soc_d[a] > soc_d[b]; });
        std::vector<int> small, large;
        const bool tiles = ctx->opt.soc_lane_entries > 0;  // 0: a warp per cone throughout
        for (int c : ord) {
            if (huge[c]) continue;
            (!tiles || soc_d[c] > kSocTileRows ? large : small).push_back(c);
        }
        t_row0.push_back(0);
        for (size_t i = 0; i < small.size();) {
            const int d0 = soc_d[small[i]];
            int lg = 0;
            const int per_lane = ctx->opt.soc_lane_entries;
            while (lg < 5 && ((32 >> lg) * d0 > kSocTileRows || d0 > (1 << lg) * per_lane)) ++lg;
            t_cone0.push_back((int)t_order.size());
            t_lg.push_back((unsigned char)lg);
            const int row0 = (int)t_trow.size();
            for (int q = 0; q < (32 >> lg) && i < small.size(); ++q, ++i) {
                const int c = small[i];
                t_order.push_back(c);
                t_so.push_back((int)t_trow.size() - row0);
                for (int r = 0; r < soc_d[c]; ++r) t_trow.push_back(soc_off_i[c] + r);
            }
            t_row0.push_back((int)t_trow.size());
        }
        t_cone0.push_back((int)t_order.size());  // the large cones start here
        for (int c : large) t_order.push_back(c);
        n_large = (int)large.size();
    }
    const int n_tiles = (int)t_lg.size();
    // the tiles are dealt round-robin over at most two blocks per SM (largest cones first),
    // so the SMs' shares of the FP64 work differ by about one tile
    const int nb_tiles = (int)std::min<long long>((n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock, 2LL * ctx->sms);
    if (ctx->opt.batch_blocks == 0 && ctx->n_soc > 0) {
        const int nb_large =
            n_large > 0 ? (int)std::min<long long>((n_large + kWarpsPerBlock - 1) / kWarpsPerBlock, (long long)ctx->sms * 8)
                        : 0;
        nb_soc = nb_tiles + nb_large;
    }
    // exp cones: one thread each, at most 256 per block but no fewer blocks than SMs
    // while each keeps a full warp (their FP64 work is bound by each SM's FP64 units)
    // exp cones: one thread each, whole warps spread evenly over the SMs (their FP64 work is
    // bound by each SM's FP64 pipe, so the SM with the most warps sets the time): up to
    // 8 * SMs warps, one block of ceil(warps / SMs) warps per SM; beyond, full blocks
    const long long exp_warps = (ctx->n_exp + kWarp - 1) / kWarp;
    const int exp_pb = (int)std::min<long long>(256, kWarp * std::max<long long>(1, (exp_warps + ctx->sms - 1) / ctx->sms));
    int nb_exp = ctx->n_exp > 0 ? (int)std::min<long long>((ctx->n_exp + exp_pb - 1) / exp_pb, (long long)ctx->sms * 8) : 0;
    ctx->g_dual = std::max(1, nb_scal + nb_soc + nb_exp);
    if (ctx->opt.batch_blocks > 0) {
        // one grid for every launch, shared by the programs of a batch: the cone roles keep
        // their share of it (at least one block each), blocks beyond the split stay idle
        const int G = ctx->opt.batch_blocks;
        ctx->g_vec_n = ctx->g_vec_m = ctx->g_kktd = ctx->g_dual = G;
        const int kinds = (nb_scal > 0) + (nb_soc > 0) + (nb_exp > 0);
        const int tot = nb_scal + nb_soc + nb_exp;
        if (tot > G) {
            auto share = [&](int nb) { return nb > 0 ? std::max(1, (int)((long long)nb * (G - kinds) / tot)) : 0; };
            nb_exp = share(nb_exp);
            nb_soc = share(nb_soc);
            nb_scal = share(nb_scal);
        }
    }
    // the team blocks' partial slots follow the role blocks (dual update, FP64 iterates) and
    // kkt_primal's blocks (checks)
    const int team_gb0 = nb_scal + nb_soc + nb_exp;
    // the K' product with the primal update's epilogue (sliced storage, single programs):
    // its blocks write their ||dx||^2 partials after primal_update's
    ctx->fuse_primal = sliced && ctx->opt.batch_blocks == 0 && ctx->opt.fuse_primal != 0;
    const int kt_grid = (int)((hkt.long_row.size() + kWarpsPerBlock - 1) / kWarpsPerBlock +
                              (std::max<size_t>(hkt.slice_off.size(), 1) - 1 + kWarpsPerBlock - 1) / kWarpsPerBlock);
    PartLayout pl;
    pl.primal_blocks = ctx->g_vec_n + (ctx->fuse_primal ? kt_grid : 0) + (n_pc > 0 ? n_pc * pc_nch : 0);
    pl.dual_blocks = team_nb > 0 ? team_gb0 + team_nb : ctx->g_dual;
    pl.kktp_blocks = ctx->g_dual + team_nb;
    pl.kktd_blocks = ctx->g_kktd;
    pl.off_px = 0;
    pl.off_dy = pl.off_px + pl.primal_blocks;
    pl.off_kp = pl.off_dy + 2LL * pl.dual_blocks;
    pl.off_kd = pl.off_kp + 2LL * kKktPN * pl.kktp_blocks;
    pl.total = pl.off_kd + 2LL * kKktDN * pl.kktd_blocks;

    Arena& A = ctx->arena;
    A.reserve<int>(m + 1); A.reserve<int>(nnz); A.reserve<int>(n + 1); A.reserve<int>(nnz);
    A.reserve<int>(m + 1); A.reserve<int>(n + 1);                    // SpMV row lists
    A.reserve<int>(m + 1); A.reserve<int>(eK); A.reserve<int>(n + 1); A.reserve<int>(eKT);  // SpMV rp, ci
    A.reserve<double>(eK); A.reserve<double>(eKT);                   // val0, val0T (then the SpMV values)
    A.reserve<double>(nnz); A.reserve<double>(nnz);                  // val, valT
    for (const SliceHost* H : {&hk, &hkt}) {                         // sliced plans
        A.reserve<int>(H->slice_off.size() + 1); A.reserve<int>(H->out_row.size() + 1);
        A.reserve<unsigned char>(H->slice_lg.size() + 1);
        A.reserve<int>(H->long_row.size() + 1); A.reserve<int>(H->long_rp.size() + 1);
    }
    for (int k = 0; k < 4; ++k) A.reserve<double>(n);                // c0 l0 u0 + cs
    A.reserve<double>(m); A.reserve<double>(m);                      // h0, hs
    A.reserve<double>(n); A.reserve<double>(n);                      // ls us
    A.reserve<double>(m); A.reserve<double>(n); A.reserve<double>(m); A.reserve<double>(n);  // dr dc rn cn
    A.reserve<int>(ctx->n_soc + 1); A.reserve<int>(ctx->n_soc + 1); A.reserve<unsigned char>(ctx->n_soc + 1);
    A.reserve<int>(ctx->n_tie + 1); A.reserve<int>(ctx->n_tie + 1);
    A.reserve<float>(ctx->n_soc + 1); A.reserve<float>(ctx->n_exp + 1);
    A.reserve<int>(t_cone0.size() + 1); A.reserve<int>(t_row0.size() + 1); A.reserve<unsigned char>(t_lg.size() + 1);
    A.reserve<int>(t_order.size() + 1); A.reserve<int>(t_trow.size() + 1); A.reserve<int>(t_so.size() + 1);
    const int n_team = (int)team_cone.size();
    for (int k = 0; k < 3; ++k) A.reserve<int>(n_team + 1);          // team_cone, team_b0, team_g
    A.reserve<unsigned>(2LL * n_team + 2); A.reserve<double>(2LL * team_nb * kTeamQ + 1);
    A.reserve<unsigned char>(ctx->n_soc + 1);                         // soc_huge
    A.reserve<unsigned char>(ctx->n_exp + 1);                         // exp_kind
    A.reserve<double>(m); A.reserve<double>(m); A.reserve<double>(3LL * ctx->n_exp + 1);
    A.reserve<double>(pl.total);
    A.reserve<Ctrl>(1);
    A.reserve<double>(16);
    for (int k = 0; k < 8; ++k) A.reserve<double>(n);  // x xh x0 kty ktyh kty0 xsum xh1
    for (int k = 0; k < 8; ++k) A.reserve<double>(m);  // y yh y0 kx kxh0 kxh1 kx0 ysum
    A.reserve<double>(2LL * n); A.reserve<double>(2LL * m); A.reserve<double>(2LL * m); A.reserve<double>(2LL * n);
    A.reserve<double>(2LL * m);  // scr
    const bool f32 = ctx->opt.precision == PDCS_PRECISION_FP32;
    if (f32) {
        A.reserve<float>(eK); A.reserve<float>(eKT);                     // val_f, valT_f
        for (int k = 0; k < 3; ++k) A.reserve<float>(n);                 // c l u
        A.reserve<float>(m);                                             // h
        for (int k = 0; k < 8; ++k) A.reserve<float>(n);                 // x xh x0 kty ktyh kty0 xsum xh1
        for (int k = 0; k < 8; ++k) A.reserve<float>(m);                 // y yh y0 kx kxh0 kxh1 kx0 ysum
        A.reserve<float>(m); A.reserve<float>(3LL * ctx->n_exp + 1);      // soc_w32, exp_lg32
    }
    if (ctx->opt.exp_mlp) A.reserve<float>(kExpMlpParams);
    A.reserve<int>(n_pc + 1); A.reserve<int>(n_pc + 1); A.reserve<unsigned char>(n_pc + 1);  // pc_off dim rot
    A.reserve<double>(2LL * n_pc * pc_nch + 1); A.reserve<double>(2LL * n_pc + 1);            // pc_ss, pc_t
    A.reserve<double>(2LL * pc_len + 1);                                                       // pc_mu
    {
        cudaError_t e = cudaMalloc(&A.base, A.plan);
        if (e != cudaSuccess) {
            ctx->err = std::string("cudaMalloc of ") + std::to_string(A.plan) + " bytes: " + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? PDCS_ERR_OOM : PDCS_ERR_CUDA;
        }
        A.cap = A.plan;
    }
    ctx->rp = A.take<int>(m + 1); ctx->ci = A.take<int>(nnz);
    ctx->rpT = A.take<int>(n + 1); ctx->ciT = A.take<int>(nnz);
    ctx->pk.list = A.take<int>(m + 1); ctx->pkt.list = A.take<int>(n + 1);
    ctx->pk.rp = A.take<int>(m + 1); ctx->pk.ci = A.take<int>(eK);
    ctx->pkt.rp = A.take<int>(n + 1); ctx->pkt.ci = A.take<int>(eKT);
    ctx->val0 = A.take<double>(eK); ctx->val0T = A.take<double>(eKT);
    ctx->val = A.take<double>(nnz); ctx->valT = A.take<double>(nnz);
    {
        SpmvPlan* PP[2] = {&ctx->pk, &ctx->pkt};
        const SliceHost* HH[2] = {&hk, &hkt};
        for (int k = 0; k < 2; ++k) {
            SlicePlan& S = PP[k]->S;
            const SliceHost& H = *HH[k];
            S.slice_off = A.take<int>(H.slice_off.size() + 1);
            S.out_row = A.take<int>(H.out_row.size() + 1);
            S.slice_lg = A.take<unsigned char>(H.slice_lg.size() + 1);
            S.long_row = A.take<int>(H.long_row.size() + 1);
            S.long_rp = A.take<int>(H.long_rp.size() + 1);
            S.nslices = H.slice_off.empty() ? 0 : (int)H.slice_off.size() - 1;
            S.nlong = (int)H.long_row.size();
            S.nb_long = (S.nlong + kWarpsPerBlock - 1) / kWarpsPerBlock;
            S.grid = S.nb_long + (S.nslices + kWarpsPerBlock - 1) / kWarpsPerBlock;
        }
    }
    ctx->c0 = A.take<double>(n); ctx->l0 = A.take<double>(n); ctx->u0 = A.take<double>(n); ctx->cs = A.take<double>(n);
    ctx->h0 = A.take<double>(m); ctx->hs = A.take<double>(m);
    ctx->ls = A.take<double>(n); ctx->us = A.take<double>(n);
    ctx->dr = A.take<double>(m); ctx->dc = A.take<double>(n); ctx->rn = A.take<double>(m); ctx->cn = A.take<double>(n);
    ctx->soc_off = A.take<int>(ctx->n_soc + 1); ctx->soc_dim = A.take<int>(ctx->n_soc + 1);
    ctx->soc_rot = A.take<unsigned char>(ctx->n_soc + 1);
    ctx->tie_off = A.take<int>(ctx->n_tie + 1); ctx->tie_len = A.take<int>(ctx->n_tie + 1);
    ctx->soc_lam = A.take<float>(ctx->n_soc + 1); ctx->exp_L = A.take<float>(ctx->n_exp + 1);
    int* d_tcone0 = A.take<int>(t_cone0.size() + 1);
    int* d_trow0 = A.take<int>(t_row0.size() + 1);
    unsigned char* d_tlg = A.take<unsigned char>(t_lg.size() + 1);
    int* d_order = A.take<int>(t_order.size() + 1);
    int* d_trow = A.take<int>(t_trow.size() + 1);
    int* d_so = A.take<int>(t_so.size() + 1);
    int* d_team_cone = A.take<int>(n_team + 1);
    int* d_team_b0 = A.take<int>(n_team + 1);
    int* d_team_g = A.take<int>(n_team + 1);
    unsigned* d_team_bar = A.take<unsigned>(2LL * n_team + 2);
    double* d_team_part = A.take<double>(2LL * team_nb * kTeamQ + 1);
    unsigned char* d_huge = A.take<unsigned char>(ctx->n_soc + 1);
    unsigned char* d_exp_kind = A.take<unsigned char>(ctx->n_exp + 1);
    ctx->soc_w = A.take<double>(m); ctx->soc_wp = A.take<double>(m); ctx->exp_lg = A.take<double>(3LL * ctx->n_exp + 1);
    ctx->part = A.take<double>(pl.total);
    ctx->ctrl = A.take<Ctrl>(1);
    ctx->scal = A.take<double>(16);
    Dev<double>& D = ctx->D;
    D.x = A.take<double>(n); D.xh = A.take<double>(n); D.x0 = A.take<double>(n); D.kty = A.take<double>(n);
    D.ktyh = A.take<double>(n); D.kty0 = A.take<double>(n); D.xsum = A.take<double>(n); D.xh1 = A.take<double>(n);
    D.y = A.take<double>(m); D.yh = A.take<double>(m); D.y0 = A.take<double>(m); D.kx = A.take<double>(m);
    D.kxh0 = A.take<double>(m); D.kxh1 = A.take<double>(m); D.kx0 = A.take<double>(m); D.ysum = A.take<double>(m);
    D.xc = A.take<double>(2LL * n); D.yc = A.take<double>(2LL * m); D.kxc = A.take<double>(2LL * m);
    D.ktyc = A.take<double>(2LL * n); D.scr = A.take<double>(2LL * m);
    int* d_pc_off = A.take<int>(n_pc + 1);
    int* d_pc_dim = A.take<int>(n_pc + 1);
    unsigned char* d_pc_rot = A.take<unsigned char>(n_pc + 1);
    D.pc_ss = A.take<double>(2LL * n_pc * pc_nch + 1);
    D.pc_t = A.take<double>(2LL * n_pc + 1);
    D.pc_mu = A.take<double>(2LL * pc_len + 1);
    D.pc_off = d_pc_off; D.pc_dim = d_pc_dim; D.pc_rot = d_pc_rot;
    D.n_pc = n_pc; D.pc_lo = n_pc > 0 ? pc_o[0] : 0; D.pc_len = pc_len; D.pc_nch = pc_nch;
    D.pc_slot0 = ctx->g_vec_n;
    Dev<float>& DF = ctx->DF;
    float *c_f = nullptr, *l_f = nullptr, *u_f = nullptr, *h_f = nullptr, *soc_w32 = nullptr, *exp_lg32 = nullptr;
    if (f32) {
        ctx->val_f = A.take<float>(eK); ctx->valT_f = A.take<float>(eKT);
        c_f = A.take<float>(n); l_f = A.take<float>(n); u_f = A.take<float>(n); h_f = A.take<float>(m);
        DF.x = A.take<float>(n); DF.xh = A.take<float>(n); DF.x0 = A.take<float>(n); DF.kty = A.take<float>(n);
        DF.ktyh = A.take<float>(n); DF.kty0 = A.take<float>(n); DF.xsum = A.take<float>(n); DF.xh1 = A.take<float>(n);
        DF.y = A.take<float>(m); DF.yh = A.take<float>(m); DF.y0 = A.take<float>(m); DF.kx = A.take<float>(m);
        DF.kxh0 = A.take<float>(m); DF.kxh1 = A.take<float>(m); DF.kx0 = A.take<float>(m); DF.ysum = A.take<float>(m);
        soc_w32 = A.take<float>(m); exp_lg32 = A.take<float>(3LL * ctx->n_exp + 1);
    }
    float* exp_mlp = ctx->opt.exp_mlp ? A.take<float>(kExpMlpParams) : nullptr;

    cudaStream_t s = ctx->stream;
    CK(cudaMemsetAsync(A.base, 0, A.used, s));
    CK(cudaMemcpyAsync(ctx->rp, rp_i.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->ci, ci_i.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->rpT, rpT.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->ciT, ciT.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->val0, v_i.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->val0T, vT.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->c0, c, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->l0, l_h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->u0, u_h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->h0, h_i.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    if (exp_mlp)
        CK(cudaMemcpyAsync(exp_mlp, ctx->opt.exp_mlp, sizeof(float) * kExpMlpParams, cudaMemcpyHostToDevice, s));
    if (ctx->n_soc) {
        CK(cudaMemcpyAsync(ctx->soc_off, soc_off_i.data(), sizeof(int) * ctx->n_soc, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->soc_dim, soc_d.data(), sizeof(int) * ctx->n_soc, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->soc_rot, soc_r.data(), ctx->n_soc, cudaMemcpyHostToDevice, s));
    }
    {
        auto up = [&](void* dst, const void* srcp, size_t bytes) {
            return bytes ? cudaMemcpyAsync(dst, srcp, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
        };
        CK(up(d_tcone0, t_cone0.data(), sizeof(int) * t_cone0.size()));
        CK(up(d_trow0, t_row0.data(), sizeof(int) * t_row0.size()));
        CK(up(d_tlg, t_lg.data(), t_lg.size()));
        CK(up(d_order, t_order.data(), sizeof(int) * t_order.size()));
        CK(up(d_trow, t_trow.data(), sizeof(int) * t_trow.size()));
        CK(up(d_so, t_so.data(), sizeof(int) * t_so.size()));
        CK(up(d_team_cone, team_cone.data(), sizeof(int) * n_team));
        CK(up(d_team_b0, team_b0.data(), sizeof(int) * n_team));
        CK(up(d_team_g, team_g.data(), sizeof(int) * n_team));
        CK(up(d_huge, huge.data(), (size_t)ctx->n_soc));
        CK(up(d_exp_kind, exp_k.data(), exp_k.size()));
        CK(cudaMemsetAsync(d_team_bar, 0, sizeof(unsigned) * (2 * n_team + 2), s));
    }
    if (ctx->n_tie) {
        CK(cudaMemcpyAsync(ctx->tie_off, tie_o.data(), sizeof(int) * ctx->n_tie, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->tie_len, tie_l.data(), sizeof(int) * ctx->n_tie, cudaMemcpyHostToDevice, s));
    }
    if (n_pc > 0) {
        CK(cudaMemcpyAsync(d_pc_off, pc_o.data(), sizeof(int) * n_pc, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_pc_dim, pc_dd.data(), sizeof(int) * n_pc, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_pc_rot, pc_r.data(), (size_t)n_pc, cudaMemcpyHostToDevice, s));
    }
    // the host copies above are pageable: wait before the vectors go out of scope
    CK(cudaStreamSynchronize(s));

    // ---- diagonal rescaling: Ruiz (infinity norm) then Pock-Chambolle (alpha = 1)
    std::vector<double> ones_m(m, 1.0), ones_n(n, 1.0);
    CK(cudaMemcpyAsync(ctx->dr, ones_m.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->dc, ones_n.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    if (ctx->opt.rescale != PDCS_RESCALE_NONE) {
        const int passes = ctx->opt.ruiz_iters + (ctx->opt.pock_chambolle ? 1 : 0);
        const int gr = spmv_grid(m, 32, ctx->sms), gc = spmv_grid(n, 32, ctx->sms);
        for (int it = 0; it < passes; ++it) {
            const int kind = it >= ctx->opt.ruiz_iters ? 1 : 0;
            scaled_row_norms<<<gr, kBlock, 0, s>>>(m, ctx->rp, ctx->ci, ctx->val0, ctx->dr, ctx->dc, 1, kind, ctx->rn);
            scaled_row_norms<<<gc, kBlock, 0, s>>>(n, ctx->rpT, ctx->ciT, ctx->val0T, ctx->dc, ctx->dr, 0, kind, ctx->cn);
            if (ctx->n_tie) tie_groups<<<(ctx->n_tie + 255) / 256, 256, 0, s>>>(ctx->n_tie, ctx->tie_off, ctx->tie_len, ctx->rn);
            // the columns of a primal cone block share one factor (D^{-1} K_p = K_p)
            if (n_pc) tie_groups<<<(n_pc + 255) / 256, 256, 0, s>>>(n_pc, d_pc_off, d_pc_dim, ctx->cn);
            apply_norm<<<(m + 255) / 256, 256, 0, s>>>(m, ctx->rn, ctx->dr);
            apply_norm<<<(n + 255) / 256, 256, 0, s>>>(n, ctx->cn, ctx->dc);
        }
    }
    {
        const int gr = spmv_grid(m, 32, ctx->sms), gc = spmv_grid(n, 32, ctx->sms);
        scale_values<<<gr, kBlock, 0, s>>>(m, ctx->rp, ctx->ci, ctx->val0, ctx->dr, ctx->dc, 1, ctx->val);
        scale_values<<<gc, kBlock, 0, s>>>(n, ctx->rpT, ctx->ciT, ctx->val0T, ctx->dc, ctx->dr, 0, ctx->valT);
        scale_cols<<<(n + 255) / 256, 256, 0, s>>>(n, ctx->dc, ctx->c0, ctx->l0, ctx->u0, ctx->cs, ctx->ls, ctx->us);
        scale_rows<<<(m + 255) / 256, 256, 0, s>>>(m, ctx->dr, ctx->h0, ctx->hs);
        reduce_small<<<1, kBlock, 0, s>>>(n, ctx->cs, nullptr, 0, ctx->scal + 0);
        reduce_small<<<1, kBlock, 0, s>>>(m, ctx->hs, nullptr, 0, ctx->scal + 1);
        reduce_small<<<1, kBlock, 0, s>>>(nnz, ctx->val, nullptr, 1, ctx->scal + 2);
        CK(cudaGetLastError());
    }
    double sc[3];
    CK(cudaMemcpyAsync(sc, ctx->scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double nc = std::sqrt(sc[0]), nh = std::sqrt(sc[1]), amax = sc[2];

    // ---- K~ and K~' stored bin by bin for the SpMV plans (timed on request, in the value
    // type the iterations use); the unscaled values are dead, their memory holds the
    // binned FP64 values
    ctx->valb = ctx->val0;
    ctx->valbT = ctx->val0T;
    const bool tune = ctx->opt.spmv_autotune && ctx->opt.spmv_lanes == 0 && !sliced;
    if (sliced) {
        CK(store_sliced<double>(ctx, ctx->pk, hk, ctx->rp, ctx->ci, ctx->val, ctx->valb, true));
        CK(store_sliced<double>(ctx, ctx->pkt, hkt, ctx->rpT, ctx->ciT, ctx->valT, ctx->valbT, true));
        if (f32) {
            CK(store_sliced<float>(ctx, ctx->pk, hk, ctx->rp, ctx->ci, ctx->val, ctx->val_f, false));
            CK(store_sliced<float>(ctx, ctx->pkt, hkt, ctx->rpT, ctx->ciT, ctx->valT, ctx->valT_f, false));
        }
    } else if (tune && f32) {
        CK(tune_spmv<float>(ctx, ctx->pk, rp_i, m, ctx->rp, ctx->ci, ctx->val, ctx->val_f, ctx->DF.x, ctx->DF.kx));
        CK(tune_spmv<float>(ctx, ctx->pkt, rpT, n, ctx->rpT, ctx->ciT, ctx->valT, ctx->valT_f, ctx->DF.y,
                            ctx->DF.kty));
    } else if (tune) {
        CK(tune_spmv<double>(ctx, ctx->pk, rp_i, m, ctx->rp, ctx->ci, ctx->val, ctx->valb, D.x, D.kx));
        CK(tune_spmv<double>(ctx, ctx->pkt, rpT, n, ctx->rpT, ctx->ciT, ctx->valT, ctx->valbT, D.y, D.kty));
    }
    if (tune) {  // the lists of the tuned plans (host) for the other value type
        plan_bins(rp_i, m, ctx->pk.shift, 0, ctx->sms, list_k, ctx->pk.B);
        plan_bins(rpT, n, ctx->pkt.shift, 0, ctx->sms, list_kt, ctx->pkt.B);
    }
    if (!sliced && (!tune || f32)) {
        CK(store_binned<double>(ctx, ctx->pk, rp_i, list_k, ctx->rp, ctx->ci, ctx->val, ctx->valb, !tune));
        CK(store_binned<double>(ctx, ctx->pkt, rpT, list_kt, ctx->rpT, ctx->ciT, ctx->valT, ctx->valbT, !tune));
    }
    if (!sliced && f32 && !tune) {
        CK(store_binned<float>(ctx, ctx->pk, rp_i, list_k, ctx->rp, ctx->ci, ctx->val, ctx->val_f, false));
        CK(store_binned<float>(ctx, ctx->pkt, rpT, list_kt, ctx->rpT, ctx->ciT, ctx->valT, ctx->valT_f, false));
    }

    // ---- ||K~||_2 by power iteration (constant / plain step modes)
    double eta = amax > 0.0 ? 1.0 / amax : 1.0;
    double omega = (nc > 1e-10 && nh > 1e-10) ? nc / nh : 1.0;
    if (ctx->opt.step_mode != PDCS_STEP_ADAPTIVE) {
        double* v = D.xc;
        double* w = D.kxc;
        double* u = D.ktyc;
        std::vector<double> v0(n, 1.0 / std::sqrt((double)n));
        CK(cudaMemcpyAsync(v, v0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        double est = 0.0;
        for (int it = 0; it < ctx->opt.power_iters; ++it) {
            launch_spmv<double>(ctx->pk, s, ctx->pk.rp, ctx->pk.ci, ctx->valb, v, w, nullptr, nullptr, 0, 0);
            launch_spmv<double>(ctx->pkt, s, ctx->pkt.rp, ctx->pkt.ci, ctx->valbT, w, u, nullptr, nullptr, 0,
                                        0);
            reduce_small<<<1, kBlock, 0, s>>>(n, u, nullptr, 0, ctx->scal + 3);
            double ss;
            CK(cudaMemcpyAsync(&ss, ctx->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const double nu = std::sqrt(ss);
            if (!(nu > 0.0)) break;
            est = std::sqrt(nu);
            scale_by_inv<<<vec_grid(n, ctx->sms), kBlock, 0, s>>>(n, u, ctx->scal + 3, v);
        }
        ctx->norm2 = est;
        const double nn = est > 0.0 ? est : 1.0;
        eta = (ctx->opt.step_mode == PDCS_STEP_PLAIN ? 0.9 : 0.998) / nn;
        if (ctx->opt.step_mode == PDCS_STEP_PLAIN) omega = 1.0;
        CK(cudaMemsetAsync(D.xc, 0, sizeof(double) * 2 * n, s));
        CK(cudaMemsetAsync(D.kxc, 0, sizeof(double) * 2 * m, s));
        CK(cudaMemsetAsync(D.ktyc, 0, sizeof(double) * 2 * n, s));
    }

    // ---- device view
    D.m = m; D.n = n;
    D.rp = ctx->pk.rp; D.ci = ctx->pk.ci; D.val = ctx->valb;
    D.rpT = ctx->pkt.rp; D.ciT = ctx->pkt.ci; D.valT = ctx->valbT;
    D.c = ctx->cs; D.h = ctx->hs; D.l = ctx->ls; D.u = ctx->us; D.dr = ctx->dr; D.dc = ctx->dc;
    D.c64 = ctx->cs; D.h64 = ctx->hs; D.l64 = ctx->ls; D.u64 = ctx->us;
    D.m_zero = ctx->m_zero; D.m_scalar = ctx->m_scalar;
    D.n_soc = ctx->n_soc; D.soc_off = ctx->soc_off; D.soc_dim = ctx->soc_dim; D.soc_rot = ctx->soc_rot;
    D.soc_lam = ctx->soc_lam; D.soc_w = ctx->soc_w; D.soc_wp = ctx->soc_wp; D.exp_lg = ctx->exp_lg;
    D.exp_row0 = ctx->exp_row0; D.n_exp = ctx->n_exp; D.exp_L = ctx->exp_L;
    D.exp_kind = std::find(exp_k.begin(), exp_k.end(), (unsigned char)1) != exp_k.end() ? d_exp_kind : nullptr;
    D.nb_scal = nb_scal; D.nb_soc = nb_soc; D.nb_exp = nb_exp; D.exp_pb = exp_pb; D.nb_primal = ctx->g_vec_n;
    D.n_tiles = ctx->opt.batch_blocks == 0 ? n_tiles : 0;
    D.nb_tiles = ctx->opt.batch_blocks == 0 ? nb_tiles : 0;
    D.n_large = n_large;
    D.tile_cone0 = d_tcone0; D.tile_row0 = d_trow0; D.tile_lg = d_tlg; D.soc_order = d_order; D.soc_trow = d_trow;
    D.soc_so = d_so;
    D.team_nb = team_nb; D.n_team = n_team;
    D.team_cone = d_team_cone; D.team_b0 = d_team_b0; D.team_g = d_team_g;
    D.team_bar = d_team_bar; D.team_part = d_team_part;
    D.soc_huge = n_team > 0 ? d_huge : nullptr;
    D.team_gb0 = team_gb0; D.team_kb0 = ctx->g_dual;
    D.px_f0 = ctx->g_vec_n;
    ctx->team_cones = n_team;
    D.part = ctx->part; D.pl = pl; D.ctrl = ctx->ctrl;
    D.l_orig = ctx->l0; D.u_orig = ctx->u0;
    D.exp_mlp = exp_mlp;
    D.binsK = ctx->pk.B; D.binsKT = ctx->pkt.B; D.listK = ctx->pk.list; D.listKT = ctx->pkt.list;
    ctx->launches_per_attempt = ctx->opt.batch_blocks > 0
                                    ? kLaunchesPerAttempt
                                    : 3 + (nb_scal > 0) + (nb_soc > 0) + (nb_exp > 0) + (team_nb > 0) +
                                          (n_pc > 0 ? 2 : 0);

    // ---- controller scalars
    Ctrl C;
    std::memset(&C, 0, sizeof(C));
    C.eta = eta; C.omega = omega; C.tau = eta / omega; C.sigma = eta * omega;
    C.beta = ctx->opt.beta;
    C.phi_prev = INFINITY;
    C.hmax = hmax; C.cmax = cmax;
    C.step_mode = ctx->opt.step_mode;
    C.status = kRunning;
    *ctx->h_ctrl = C;
    CK(cudaMemcpyAsync(ctx->ctrl, ctx->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    std::vector<float> nanv(std::max(ctx->n_soc, ctx->n_exp) + 1, NAN);
    CK(cudaMemcpyAsync(ctx->exp_L, nanv.data(), sizeof(float) * (ctx->n_exp + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->soc_lam, nanv.data(), sizeof(float) * (ctx->n_soc + 1), cudaMemcpyHostToDevice, s));
    if (ctx->n_soc)
        cone_constants<<<(ctx->n_soc + kWarpsPerBlock - 1) / kWarpsPerBlock, kBlock, 0, s>>>(
            ctx->n_soc, ctx->soc_off, ctx->soc_dim, ctx->dr, ctx->soc_w, ctx->soc_wp);
    if (ctx->n_exp)
        exp_constants<<<(ctx->n_exp + 255) / 256, 256, 0, s>>>(ctx->n_exp, ctx->exp_row0, ctx->dr, ctx->exp_lg);
    if (f32) {
        const int g = vec_grid(std::max<long long>(nnz, std::max(m, n)), ctx->sms);
        cast_vec<float><<<g, kBlock, 0, s>>>(n, ctx->cs, c_f);
        cast_vec<float><<<g, kBlock, 0, s>>>(n, ctx->ls, l_f);
        cast_vec<float><<<g, kBlock, 0, s>>>(n, ctx->us, u_f);
        cast_vec<float><<<g, kBlock, 0, s>>>(m, ctx->hs, h_f);
        cast_vec<float><<<g, kBlock, 0, s>>>(m, ctx->soc_w, soc_w32);
        cast_vec<float><<<g, kBlock, 0, s>>>(3LL * ctx->n_exp, ctx->exp_lg, exp_lg32);
        // the FP32 view: FP32 matrix, data and state; everything else shared with D
        float *x = DF.x, *xh = DF.xh, *x0 = DF.x0, *kty = DF.kty, *ktyh = DF.ktyh, *kty0 = DF.kty0, *xsum = DF.xsum,
              *xh1 = DF.xh1;
        float *y = DF.y, *yh = DF.yh, *y0 = DF.y0, *kx = DF.kx, *kxh0 = DF.kxh0, *kxh1 = DF.kxh1, *kx0 = DF.kx0,
              *ysum = DF.ysum;
        static_assert(sizeof(Dev<float>) == sizeof(Dev<double>), "Dev layouts differ only in pointee types");
        std::memcpy(static_cast<void*>(&DF), static_cast<const void*>(&D), sizeof(Dev<float>));
        DF.val = ctx->val_f; DF.valT = ctx->valT_f;
        DF.c = c_f; DF.h = h_f; DF.l = l_f; DF.u = u_f;
        DF.x = x; DF.xh = xh; DF.x0 = x0; DF.kty = kty; DF.ktyh = ktyh; DF.kty0 = kty0; DF.xsum = xsum; DF.xh1 = xh1;
        DF.y = y; DF.yh = yh; DF.y0 = y0; DF.kx = kx; DF.kxh0 = kxh0; DF.kxh1 = kxh1; DF.kx0 = kx0; DF.ysum = ysum;
        DF.soc_w32 = soc_w32; DF.exp_lg32 = exp_lg32;
        ctx->fp32_active = true;
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    return PDCS_OK;
}

// One check period (attempts + check) of the running phase as a CUDA graph.
pdcs_status capture_graph(pdcs_ctx* ctx) {
    cudaGraphExec_t& G = ctx->fp32_active ? ctx->graph32 : ctx->graph;
    if (G) return PDCS_OK;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    for (int a = 0; a < ctx->opt.check_period; ++a) enqueue_attempt(ctx);
    enqueue_check(ctx);
    CK(cudaStreamEndCapture(ctx->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&G, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        G = nullptr;
        ctx->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        return PDCS_ERR_CUDA;
    }
    return PDCS_OK;
}

// FP32 phase -> FP64 phase, continuing the same trajectory and restart period: the pending
// Halpern update is applied in FP32, the iterate, the anchor and the average's sums are
// widened into the FP64 state, the cached products K~x, K~x0, K~'y, K~'y0 are formed
// afresh by the FP64 SpMV (the FP32 ones carry FP32 rounding), and every scalar of
// Algorithm 1 (step size, primal weight, inner index, weights, restart metrics) is kept.
pdcs_status switch_to_fp64(pdcs_ctx* ctx) {
    cudaStream_t s = ctx->stream;
    Dev<double>& D = ctx->D;
    Dev<float>& F = ctx->DF;
    k_flush_primal(F, ctx->g_vec_n, s);
    k_flush_dual(F, ctx->g_vec_m, s);
    clear_pending<<<1, 1, 0, s>>>(ctx->ctrl);  // the FP64 primal update forms x-hat afresh
    const int g = vec_grid(std::max(ctx->m, ctx->n), ctx->sms);
    const float* fn[3] = {F.x, F.x0, F.xsum};
    double* dn[3] = {D.x, D.x0, D.xsum};
    const float* fm[3] = {F.y, F.y0, F.ysum};
    double* dm[3] = {D.y, D.y0, D.ysum};
    for (int k = 0; k < 3; ++k) {
        widen<<<g, kBlock, 0, s>>>(ctx->n, fn[k], dn[k]);
        widen<<<g, kBlock, 0, s>>>(ctx->m, fm[k], dm[k]);
    }
    launch_spmv<double>(ctx->pk, s, D.rp, D.ci, D.val, D.x, D.kx, nullptr, nullptr, 0, 0);
    launch_spmv<double>(ctx->pk, s, D.rp, D.ci, D.val, D.x0, D.kx0, nullptr, nullptr, 0, 0);
    launch_spmv<double>(ctx->pkt, s, D.rpT, D.ciT, D.valT, D.y, D.kty, nullptr, nullptr, 0, 0);
    launch_spmv<double>(ctx->pkt, s, D.rpT, D.ciT, D.valT, D.y0, D.kty0, nullptr, nullptr, 0, 0);
    ctx->launches += 13;
    CK(cudaGetLastError());
    ctx->fp32_active = false;
    CK(cudaStreamSynchronize(s));
    return PDCS_OK;
}

// Whether the FP32 phase should hand over: the relative KKT error of the last check is
// at most fp32_switch_tol or the requested tolerance, or its best value has not improved
// by 10 % over 50 checks (the FP32 rounding floor; restarts make the error itself
// non-monotone, so the window is long).
bool fp32_done(pdcs_ctx* ctx, double tol) {
    const Ctrl& C = *ctx->h_ctrl;
    const double err = std::max(C.err[0], std::max(C.err[1], C.err[2]));
    if (!(err == err)) return false;
    if (err <= ctx->opt.fp32_switch_tol || err <= tol) return true;
    if (err < 0.9 * ctx->fp32_best) {
        ctx->fp32_best = err;
        ctx->fp32_stall = 0;
    } else if (++ctx->fp32_stall >= 50) {
        return true;
    }
    return false;
}

pdcs_status status_of(const Ctrl& C) {
    if (C.status == kConverged) return PDCS_OK;
    if (C.status == kNumericError) return PDCS_ERR_NUMERIC;
    if (C.status == kTimeout) return PDCS_ERR_DEVICE_TIMEOUT;
    return PDCS_MAX_ITER;
}

void fill_info(pdcs_ctx* ctx, pdcs_info* info) {
    const Ctrl& C = *ctx->h_ctrl;
    info->attempts = C.attempts;
    info->accepted = C.accepted;
    info->restarts = C.restarts;
    info->err_p = C.err[0];
    info->err_d = C.err[1];
    info->err_gap = C.err[2];
    info->pobj = C.pobj;
    info->dobj = C.dobj;
    info->eta = C.eta;
    info->omega = C.omega;
    info->setup_seconds = ctx->setup_seconds;
    info->solve_seconds = ctx->solve_seconds;
    info->status = ctx->last_status;
    info->fp64_phase = ctx->fp32_active ? 0 : 1;
    info->kernel_launches = ctx->launches;
    info->spmv_plan[0] = ctx->pk.shift;
    info->spmv_plan[1] = ctx->pk.unroll;
    info->spmv_plan[2] = ctx->pkt.shift;
    info->spmv_plan[3] = ctx->pkt.unroll;
    info->spmv_format = ctx->pk.format;
    info->soc_grid_cones = ctx->team_cones;
    info->fuse_primal = ctx->fuse_primal ? 1 : 0;
}

__global__ void batch_prepare(Dev<double>* views, int count, double tol, int start) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    Ctrl* C = views[i].ctrl;
    C->tol = tol;
    if (start) C->check_mode = 1;
}

__global__ void batch_status(const Dev<double>* views, int count, int* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = views[i].ctrl->status;
}

}  // namespace

// A batch: programs created with the same batch_blocks, iterated in lockstep by launches
// whose third grid dimension is the program (one CUDA graph per check period).
struct pdcs_batch {
    std::vector<pdcs_ctx*> ctxs;    // all programs
    std::vector<int> active;        // programs in the launches (those still running, compacted)
    cudaStream_t stream = nullptr;
    Dev<double>* views = nullptr;  // device copies of the programs' views
    int* d_status = nullptr;
    int* h_status = nullptr;       // pinned
    int G = 0, g_spmv = 0, period = 64;
    cudaGraphExec_t graph = nullptr;
    bool started = false;
    std::string err;
    ~pdcs_batch() {
        if (graph) cudaGraphExecDestroy(graph);
        if (views) cudaFree(views);
        if (d_status) cudaFree(d_status);
        if (h_status) cudaFreeHost(h_status);
    }
};

namespace {

void batch_attempt(pdcs_batch* b) {
    const int B = (int)b->active.size();
    cudaStream_t s = b->stream;
    k_batch(kbPrimalUpdate, b->views, dim3(b->G, 1, B), s);
    k_spmv_batch(b->views, dim3(b->g_spmv, 1, B), 0, s);
    k_batch(kbDualUpdate, b->views, dim3(b->G, 1, B), s);
    k_spmv_batch(b->views, dim3(b->g_spmv, 1, B), 1, s);
    for (int i : b->active) b->ctxs[i]->launches += kLaunchesPerAttempt;
}

void batch_check(pdcs_batch* b) {
    const int B = (int)b->active.size();
    cudaStream_t s = b->stream;
    k_batch(kbFlushPrimal, b->views, dim3(b->G, 1, B), s);
    k_batch(kbFlushDual, b->views, dim3(b->G, 1, B), s);
    k_batch(kbCandPrimal, b->views, dim3(b->G, 2, B), s);
    k_batch(kbCandDual, b->views, dim3(b->G, 2, B), s);
    k_spmv_batch(b->views, dim3(b->g_spmv, 2, B), 2, s);
    k_spmv_batch(b->views, dim3(b->g_spmv, 2, B), 3, s);
    k_batch(kbKktPrimal, b->views, dim3(b->G, 2, B), s);
    k_batch(kbKktDual, b->views, dim3(b->G, 1, B), s);
    k_batch(kbRestartPrimal, b->views, dim3(b->G, 1, B), s);
    k_batch(kbRestartDual, b->views, dim3(b->G, 1, B), s);
    for (int i : b->active) b->ctxs[i]->launches += kLaunchesPerCheck;
}

#define CKB(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            b->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return e_ == cudaErrorMemoryAllocation ? PDCS_ERR_OOM : PDCS_ERR_CUDA;       \
        }                                                                                \
    } while (0)

// Status of every program in the launches (h_status, in the order of `active`).
pdcs_status batch_read(pdcs_batch* b) {
    const int B = (int)b->active.size();
    batch_status<<<(B + 255) / 256, 256, 0, b->stream>>>(b->views, B, b->d_status);
    CKB(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int) * B, cudaMemcpyDeviceToHost, b->stream));
    CKB(cudaStreamSynchronize(b->stream));
    return PDCS_OK;
}

// Keeps only the running programs in the launches (their views moved to the front),
// once at most half of the launched ones still run; the graph is captured again.
// Each program's arithmetic does not depend on the others, so results are unchanged.
pdcs_status batch_compact(pdcs_batch* b) {
    std::vector<int> keep;
    for (size_t k = 0; k < b->active.size(); ++k)
        if (b->h_status[k] == kRunning) keep.push_back(b->active[k]);
    if (keep.empty() || keep.size() * 2 > b->active.size()) return PDCS_OK;
    std::vector<Dev<double>> hv(keep.size());
    b->g_spmv = 1;
    for (size_t k = 0; k < keep.size(); ++k) {
        const pdcs_ctx* c = b->ctxs[keep[k]];
        hv[k] = c->D;
        b->g_spmv = std::max({b->g_spmv, c->pk.B.blk[c->pk.B.nbins], c->pkt.B.blk[c->pkt.B.nbins]});
    }
    CKB(cudaMemcpyAsync(b->views, hv.data(), sizeof(Dev<double>) * keep.size(), cudaMemcpyHostToDevice, b->stream));
    CKB(cudaStreamSynchronize(b->stream));
    b->active = keep;
    for (size_t k = 0; k < keep.size(); ++k) b->h_status[k] = kRunning;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return PDCS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void pdcs_default_options(pdcs_options* o) {
    if (!o) return;
    o->rescale = PDCS_RESCALE_COORD;
    o->ruiz_iters = 10;
    o->pock_chambolle = 1;
    o->step_mode = PDCS_STEP_ADAPTIVE;
    o->check_period = 64;
    o->beta = 1.0;
    o->power_iters = 50;
    o->precision = PDCS_PRECISION_FP64;
    o->fp32_switch_tol = 1e-4;
    o->use_graphs = 1;
    o->spmv_lanes = 0;
    o->time_limit = 0.0;
    o->spmv_autotune = 0;
    o->exp_mlp = nullptr;
    o->batch_blocks = 0;
    o->spmv_format = 0;
    o->soc_lane_entries = 0;
    o->soc_grid_dim = 0;
    o->fuse_primal = 0;
    o->primal_cones = nullptr;
    o->n_primal_cones = 0;
    o->primal_cone_start = 0;
}

pdcs_status pdcs_create(const pdcs_csr* K, const double* c, const double* h, const double* lb, const double* ub,
                        const pdcs_cone* cones, int64_t n_cones, const pdcs_options* opt, void* cuda_stream,
                        pdcs_ctx** out) {
    const double t0 = now_s();
    if (!out) { g_create_error = "out is NULL"; return PDCS_ERR_INVALID; }
    *out = nullptr;
    auto bad = [&](const std::string& s) { g_create_error = s; return PDCS_ERR_INVALID; };
    if (!K || !c || !h || !cones) return bad("K, c, h and cones are required");
    if (K->m < 1 || K->n < 1 || K->m > 0x7fffffff || K->n > 0x7fffffff) return bad("m and n must be in [1, 2^31)");
    if (!K->row_ptr || (K->nnz > 0 && (!K->col || !K->val))) return bad("CSR arrays are NULL");
    if (K->nnz < 0 || K->nnz >= 0x7fffffffLL) return bad("nnz must be in [0, 2^31)");
    if (K->row_ptr[0] != 0 || K->row_ptr[K->m] != K->nnz) return bad("row_ptr[0] must be 0 and row_ptr[m] == nnz");
    for (int64_t i = 0; i < K->m; ++i)
        if (K->row_ptr[i + 1] < K->row_ptr[i]) return bad("row_ptr is not nondecreasing");
    for (int64_t p = 0; p < K->nnz; ++p) {
        if (K->col[p] < 0 || K->col[p] >= K->n) return bad("column index out of range");
        if (!std::isfinite(K->val[p])) return bad("matrix value is NaN or Inf");
    }
    for (int64_t j = 0; j < K->n; ++j) if (!std::isfinite(c[j])) return bad("c has NaN or Inf");
    for (int64_t i = 0; i < K->m; ++i) if (!std::isfinite(h[i])) return bad("h has NaN or Inf");
    if (!finite_all(lb, K->n) || !finite_all(ub, K->n)) return bad("bounds contain NaN");
    for (int64_t j = 0; j < K->n; ++j) {
        const double l = lb ? lb[j] : 0.0, u = ub ? ub[j] : INFINITY;
        if (l > u) return bad("lb > ub");
        if (l == INFINITY || u == -INFINITY) return bad("infeasible infinite bound");
    }
    if (n_cones < 1) return bad("the cone list is empty");
    long long tot = 0;
    for (int64_t k = 0; k < n_cones; ++k) {
        const int t = cones[k].type;
        const long long d = cones[k].dim;
        if (t < PDCS_CONE_ZERO || t > PDCS_CONE_EXP_DUAL) return bad("unknown cone type");
        if (d < 1 || ((t == PDCS_CONE_EXP || t == PDCS_CONE_EXP_DUAL) && d != 3) || (t == PDCS_CONE_RSOC && d < 2))
            return bad("bad cone dimension");
        tot += d;
    }
    if (tot != K->m) return bad("cone dimensions do not sum to m");
    pdcs_options o;
    pdcs_default_options(&o);
    if (opt) o = *opt;
    if (o.check_period < 1 || o.ruiz_iters < 0 || o.power_iters < 1 || o.rescale < 0 || o.rescale > 2 ||
        o.step_mode < 0 || o.step_mode > 2 || !(o.beta >= 0.0) || o.beta > 1.0)
        return bad("invalid options");
    if (o.precision != PDCS_PRECISION_FP64 && o.precision != PDCS_PRECISION_FP32) return bad("unknown precision");
    if (!(o.fp32_switch_tol >= 0.0)) return bad("fp32_switch_tol must be >= 0");
    if (o.spmv_lanes != 0 && (o.spmv_lanes > 32 || (o.spmv_lanes & (o.spmv_lanes - 1)) != 0))
        return bad("spmv_lanes must be 0 or a power of two <= 32");
    if (o.spmv_autotune != 0 && o.spmv_autotune != 1) return bad("spmv_autotune must be 0 or 1");
    if (o.batch_blocks < 0 || o.batch_blocks > 1 << 20) return bad("batch_blocks must be in [0, 2^20]");
    if (o.spmv_format < 0 || o.spmv_format > 2) return bad("spmv_format must be 0, 1 or 2");
    if (o.soc_lane_entries < 0 || o.soc_lane_entries > 256) return bad("soc_lane_entries must be in [0, 256]");
    if (o.soc_grid_dim < -1) return bad("soc_grid_dim must be -1, 0 or positive");
    if (o.fuse_primal != 0 && o.fuse_primal != 1) return bad("fuse_primal must be 0 or 1");
    if (o.spmv_format == 2 && (o.batch_blocks > 0 || o.spmv_lanes != 0))
        return bad("the sliced SpMV format serves single programs with spmv_lanes = 0");
    if (o.n_primal_cones < 0 || (o.n_primal_cones > 0 && !o.primal_cones)) return bad("bad primal cone list");
    if (o.n_primal_cones > 0) {
        if (o.precision != PDCS_PRECISION_FP64 || o.batch_blocks > 0 || o.fuse_primal)
            return bad("primal cones need FP64 iterates, a single program and separate primal updates");
        long long pt = 0;
        for (int64_t k = 0; k < o.n_primal_cones; ++k) {
            const int t = o.primal_cones[k].type;
            const long long d = o.primal_cones[k].dim;
            if ((t != PDCS_CONE_SOC && t != PDCS_CONE_RSOC) || d < (t == PDCS_CONE_RSOC ? 2 : 1))
                return bad("primal cones are SOC (dim >= 1) or RSOC (dim >= 2)");
            pt += d;
        }
        if (o.primal_cone_start < 0 || o.primal_cone_start + pt > K->n) return bad("primal cones exceed n");
        for (long long j = o.primal_cone_start; j < o.primal_cone_start + pt; ++j)
            if (!lb || !ub || lb[j] != -INFINITY || ub[j] != INFINITY)
                return bad("primal cone variables must have lb = -inf and ub = +inf");
    }

    pdcs_ctx* ctx = new (std::nothrow) pdcs_ctx();
    if (!ctx) return bad("host allocation failed");
    ctx->opt = o;
    if (o.n_primal_cones > 0) ctx->pcones.assign(o.primal_cones, o.primal_cones + o.n_primal_cones);
    ctx->pc_start = o.primal_cone_start;
    ctx->opt.primal_cones = nullptr;  // copied; the caller's array need not outlive this call
    ctx->m = (int)K->m;
    ctx->n = (int)K->n;
    ctx->nnz = K->nnz;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            ctx->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_ctrl, sizeof(Ctrl));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&ctx->aux[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        g_create_error = std::string("CUDA setup: ") + cudaGetErrorString(e);
        delete ctx;
        return PDCS_ERR_CUDA;
    }
    if (e == cudaSuccess) e = k_prepare(static_cast<const Dev<double>*>(nullptr));
    if (e == cudaSuccess) e = k_prepare(static_cast<const Dev<float>*>(nullptr));
    if (e != cudaSuccess) {
        g_create_error = std::string("kernel attributes: ") + cudaGetErrorString(e);
        delete ctx;
        return PDCS_ERR_CUDA;
    }
    pdcs_status st = build(ctx, K, c, h, lb, ub, cones, n_cones);
    if (st != PDCS_OK) {
        g_create_error = ctx->err;
        delete ctx;
        return st;
    }
    ctx->setup_seconds = now_s() - t0;
    *out = ctx;
    return PDCS_OK;
}

pdcs_status pdcs_solve(pdcs_ctx* ctx, double tol, int64_t max_iter, pdcs_info* info) {
    if (!ctx) return PDCS_ERR_INVALID;
    if (max_iter < 0) { ctx->err = "max_iter < 0"; return PDCS_ERR_INVALID; }
    const double t0 = now_s();
    pdcs_status st = read_ctrl(ctx);
    if (st != PDCS_OK) return st;
    if (ctx->h_ctrl->status == kConverged && tol > 0.0 && tol < ctx->h_ctrl->tol) {
        // converged to a looser tolerance: continue from the same state towards the new one
        const int running = kRunning;
        CK(cudaMemcpyAsync(&ctx->ctrl->status, &running, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        ctx->h_ctrl->status = kRunning;
    }
    if (ctx->h_ctrl->status != kRunning) {  // otherwise a converged solver stays converged
        ctx->last_status = status_of(*ctx->h_ctrl);
        if (info) fill_info(ctx, info);
        return (pdcs_status)ctx->last_status;
    }
    CK(cudaMemcpyAsync(&ctx->ctrl->tol, &tol, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (!ctx->started) {
        const int one = 1;
        CK(cudaMemcpyAsync(&ctx->ctrl->check_mode, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        enqueue_check(ctx);
        CK(cudaGetLastError());
        ctx->started = true;
    }
    const int period = ctx->opt.check_period;
    long long done = ctx->h_ctrl->attempts;
    long long remaining = max_iter;
    pdcs_status result = PDCS_MAX_ITER;
    while (remaining > 0) {
        const long long to_b = period - (done % period);
        if (remaining >= to_b) {
            if (to_b == period && ctx->opt.use_graphs) {
                st = capture_graph(ctx);
                if (st != PDCS_OK) return st;
                CK(cudaGraphLaunch(ctx->fp32_active ? ctx->graph32 : ctx->graph, ctx->stream));
                ctx->launches += (long long)period * ctx->launches_per_attempt + kLaunchesPerCheck;
            } else {
                for (long long a = 0; a < to_b; ++a) enqueue_attempt(ctx);
                enqueue_check(ctx);
            }
            done += to_b;
            remaining -= to_b;
        } else {
            for (long long a = 0; a < remaining; ++a) enqueue_attempt(ctx);
            done += remaining;
            remaining = 0;
        }
        CK(cudaGetLastError());
        st = read_ctrl(ctx);
        if (st != PDCS_OK) return st;
        const bool at_check = done % period == 0;
        if (ctx->h_ctrl->status != kRunning) break;
        if (ctx->fp32_active && at_check && fp32_done(ctx, tol)) {
            st = switch_to_fp64(ctx);
            if (st != PDCS_OK) return st;
            st = read_ctrl(ctx);
            if (st != PDCS_OK) return st;
            if (ctx->h_ctrl->status != kRunning) break;
        }
        if (ctx->opt.time_limit > 0.0 && now_s() - t0 > ctx->opt.time_limit) { result = PDCS_TIME_LIMIT; break; }
    }
    st = read_ctrl(ctx);
    if (st != PDCS_OK) return st;
    if (ctx->h_ctrl->status == kConverged) result = PDCS_OK;
    else if (ctx->h_ctrl->status == kNumericError) result = PDCS_ERR_NUMERIC;
    else if (ctx->h_ctrl->status == kTimeout) result = PDCS_ERR_DEVICE_TIMEOUT;
    else if (result != PDCS_TIME_LIMIT) result = PDCS_MAX_ITER;
    if (result == PDCS_ERR_NUMERIC) ctx->err = "NaN or Inf in the iterates";
    if (result == PDCS_ERR_DEVICE_TIMEOUT) ctx->err = "a bounded wait of the grid-wise SOC projection gave up";
    ctx->solve_seconds += now_s() - t0;
    ctx->last_status = result;
    if (info) fill_info(ctx, info);
    return result;
}

static pdcs_status unscale_out(pdcs_ctx* ctx, const double* dx, const double* dy, double* x, double* y) {
    std::vector<double> hx(ctx->n), hy(ctx->m), hdc(ctx->n), hdr(ctx->m);
    CK(cudaMemcpyAsync(hdc.data(), ctx->dc, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hdr.data(), ctx->dr, sizeof(double) * ctx->m, cudaMemcpyDeviceToHost, ctx->stream));
    if (x) CK(cudaMemcpyAsync(hx.data(), dx, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    if (y) CK(cudaMemcpyAsync(hy.data(), dy, sizeof(double) * ctx->m, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (x) for (int j = 0; j < ctx->n; ++j) x[j] = hx[j] * hdc[j];
    if (y) for (int r = 0; r < ctx->m; ++r) y[ctx->perm[r]] = hy[r] * hdr[r];
    return PDCS_OK;
}

pdcs_status pdcs_get_solution(pdcs_ctx* ctx, double* x, double* y, double* lambda) {
    if (!ctx) return PDCS_ERR_INVALID;
    if (!ctx->started) { ctx->err = "no solution before the first pdcs_solve"; return PDCS_ERR_INVALID; }
    pdcs_status st = read_ctrl(ctx);
    if (st != PDCS_OK) return st;
    const int q = ctx->h_ctrl->sol_cand;
    const double* dx = ctx->D.xc + (size_t)q * ctx->n;
    const double* dy = ctx->D.yc + (size_t)q * ctx->m;
    st = unscale_out(ctx, dx, dy, x, y);
    if (st != PDCS_OK) return st;
    if (lambda) {
        std::vector<double> kt(ctx->n), cs(ctx->n), dc(ctx->n);
        CK(cudaMemcpyAsync(kt.data(), ctx->D.ktyc + (size_t)q * ctx->n, sizeof(double) * ctx->n,
                           cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(cs.data(), ctx->cs, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(dc.data(), ctx->dc, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        for (int j = 0; j < ctx->n; ++j) lambda[j] = (cs[j] - kt[j]) / dc[j];
    }
    return PDCS_OK;
}

pdcs_status pdcs_get_iterate(pdcs_ctx* ctx, double* x, double* y, double* xhat, double* yhat) {
    if (!ctx) return PDCS_ERR_INVALID;
    // materialise a pending Halpern update (same arithmetic as the next evaluation would apply)
    if (ctx->fp32_active) {
        k_flush_primal(ctx->DF, ctx->g_vec_n, ctx->stream);
        k_flush_dual(ctx->DF, ctx->g_vec_m, ctx->stream);
        xhat_first<float><<<ctx->g_vec_n, kBlock, 0, ctx->stream>>>(ctx->n, ctx->DF.xh, ctx->DF.xh1, ctx->ctrl);
    } else {
        k_flush_primal(ctx->D, ctx->g_vec_n, ctx->stream);
        k_flush_dual(ctx->D, ctx->g_vec_m, ctx->stream);
        xhat_first<double><<<ctx->g_vec_n, kBlock, 0, ctx->stream>>>(ctx->n, ctx->D.xh, ctx->D.xh1, ctx->ctrl);
    }
    clear_pending<<<1, 1, 0, ctx->stream>>>(ctx->ctrl);
    ctx->launches += 3;
    CK(cudaGetLastError());
    if (ctx->fp32_active) {  // FP32 state widened into the FP64 check scratch, then unscaled
        double* tx = ctx->D.xc + ctx->n;  // second candidate slots, rewritten by every check
        double* ty = ctx->D.yc + ctx->m;
        const int g = vec_grid(std::max(ctx->m, ctx->n), ctx->sms);
        pdcs_status st = PDCS_OK;
        const float* src[2][2] = {{ctx->DF.x, ctx->DF.y}, {ctx->DF.xh, ctx->DF.yh}};
        double* dst[2][2] = {{x, y}, {xhat, yhat}};
        for (int k = 0; k < 2 && st == PDCS_OK; ++k) {
            widen<<<g, kBlock, 0, ctx->stream>>>(ctx->n, src[k][0], tx);
            widen<<<g, kBlock, 0, ctx->stream>>>(ctx->m, src[k][1], ty);
            CK(cudaGetLastError());
            st = unscale_out(ctx, tx, ty, dst[k][0], dst[k][1]);
        }
        return st;
    }
    pdcs_status st = unscale_out(ctx, ctx->D.x, ctx->D.y, x, y);
    if (st != PDCS_OK) return st;
    return unscale_out(ctx, ctx->D.xh, ctx->D.yh, xhat, yhat);
}

pdcs_status pdcs_get_scaling(pdcs_ctx* ctx, double* dr, double* dc) {
    if (!ctx) return PDCS_ERR_INVALID;
    std::vector<double> hdr(ctx->m);
    CK(cudaMemcpyAsync(hdr.data(), ctx->dr, sizeof(double) * ctx->m, cudaMemcpyDeviceToHost, ctx->stream));
    if (dc) CK(cudaMemcpyAsync(dc, ctx->dc, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (dr) for (int r = 0; r < ctx->m; ++r) dr[ctx->perm[r]] = hdr[r];
    return PDCS_OK;
}

pdcs_status pdcs_get_info(pdcs_ctx* ctx, pdcs_info* info) {
    if (!ctx || !info) return PDCS_ERR_INVALID;
    pdcs_status st = read_ctrl(ctx);
    if (st != PDCS_OK) return st;
    fill_info(ctx, info);
    return PDCS_OK;
}

pdcs_status pdcs_set_warm_start(pdcs_ctx* ctx, const double* x, const double* y, double omega) {
    if (!ctx) return PDCS_ERR_INVALID;
    if (x) for (int j = 0; j < ctx->n; ++j) if (!std::isfinite(x[j])) { ctx->err = "x has NaN/Inf"; return PDCS_ERR_INVALID; }
    if (y) for (int i = 0; i < ctx->m; ++i) if (!std::isfinite(y[i])) { ctx->err = "y has NaN/Inf"; return PDCS_ERR_INVALID; }
    std::vector<double> hdc(ctx->n), hdr(ctx->m), xs(ctx->n, 0.0), ys(ctx->m, 0.0);
    CK(cudaMemcpyAsync(hdc.data(), ctx->dc, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hdr.data(), ctx->dr, sizeof(double) * ctx->m, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (x) for (int j = 0; j < ctx->n; ++j) xs[j] = x[j] / hdc[j];
    if (y) for (int r = 0; r < ctx->m; ++r) ys[r] = y[ctx->perm[r]] / hdr[r];
    Dev<double>& D = ctx->D;
    cudaStream_t s = ctx->stream;
    CK(cudaMemcpyAsync(D.x, xs.data(), sizeof(double) * ctx->n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.x0, xs.data(), sizeof(double) * ctx->n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.y, ys.data(), sizeof(double) * ctx->m, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.y0, ys.data(), sizeof(double) * ctx->m, cudaMemcpyHostToDevice, s));
    // cached products of the start: K x, K'y
    launch_spmv<double>(ctx->pk, s, D.rp, D.ci, D.val, D.x, D.kx, nullptr, nullptr, 0, 0);
    launch_spmv<double>(ctx->pkt, s, D.rpT, D.ciT, D.valT, D.y, D.kty, nullptr, nullptr, 0, 0);
    CK(cudaMemcpyAsync(D.kx0, D.kx, sizeof(double) * ctx->m, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(D.kty0, D.kty, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(D.xsum, 0, sizeof(double) * ctx->n, s));
    CK(cudaMemsetAsync(D.ysum, 0, sizeof(double) * ctx->m, s));
    ctx->fp32_active = ctx->opt.precision == PDCS_PRECISION_FP32;
    if (ctx->fp32_active) {  // the FP32 phase starts again, from the same point
        Dev<float>& F = ctx->DF;
        const int g = vec_grid(std::max(ctx->m, ctx->n), ctx->sms);
        cast_vec<float><<<g, kBlock, 0, s>>>(ctx->n, D.x, F.x);
        cast_vec<float><<<g, kBlock, 0, s>>>(ctx->n, D.x, F.x0);
        cast_vec<float><<<g, kBlock, 0, s>>>(ctx->m, D.y, F.y);
        cast_vec<float><<<g, kBlock, 0, s>>>(ctx->m, D.y, F.y0);
        cast_vec<float><<<g, kBlock, 0, s>>>(ctx->m, D.kx, F.kx);
        cast_vec<float><<<g, kBlock, 0, s>>>(ctx->m, D.kx, F.kx0);
        cast_vec<float><<<g, kBlock, 0, s>>>(ctx->n, D.kty, F.kty);
        cast_vec<float><<<g, kBlock, 0, s>>>(ctx->n, D.kty, F.kty0);
        CK(cudaMemsetAsync(F.xsum, 0, sizeof(float) * ctx->n, s));
        CK(cudaMemsetAsync(F.ysum, 0, sizeof(float) * ctx->m, s));
        CK(cudaGetLastError());
        ctx->fp32_best = INFINITY;
        ctx->fp32_stall = 0;
    }
    CK(cudaStreamSynchronize(s));
    pdcs_status st = read_ctrl(ctx);
    if (st != PDCS_OK) return st;
    Ctrl C = *ctx->h_ctrl;
    if (omega > 0.0) C.omega = omega;
    C.tau = C.eta / C.omega;
    C.sigma = C.eta * C.omega;
    C.pending = 0; C.wsum = 0.0; C.k = 0; C.accepted = 0; C.attempts = 0; C.restarts = 0;
    C.status = kRunning; C.check_mode = 0; C.phi_prev = INFINITY;
    C.xnext = 0;  // the next primal update forms x-hat from the new start
    *ctx->h_ctrl = C;
    CK(cudaMemcpyAsync(ctx->ctrl, ctx->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    ctx->started = false;
    return PDCS_OK;
}

pdcs_status pdcs_get_state(pdcs_ctx* ctx, pdcs_state* st, const pdcs_state_arrays* arr) {
    if (!ctx) return PDCS_ERR_INVALID;
    if (ctx->fp32_active) { ctx->err = "pdcs_get_state needs the FP64 phase"; return PDCS_ERR_INVALID; }
    cudaStream_t s = ctx->stream;
    Dev<double>& D = ctx->D;
    // apply a pending Halpern update (the arithmetic of the next evaluation's update)
    k_flush_primal(D, ctx->g_vec_n, s);
    k_flush_dual(D, ctx->g_vec_m, s);
    xhat_first<double><<<ctx->g_vec_n, kBlock, 0, s>>>(ctx->n, D.xh, D.xh1, ctx->ctrl);
    clear_pending<<<1, 1, 0, s>>>(ctx->ctrl);
    ctx->launches += 4;
    CK(cudaGetLastError());
    pdcs_status r = read_ctrl(ctx);
    if (r != PDCS_OK) return r;
    if (arr) {
        const int n = ctx->n, m = ctx->m;
        const double* srcn[6] = {D.x, D.xh, D.x0, D.xsum, D.kty, D.kty0};
        double* dstn[6] = {arr->x, arr->xhat, arr->x0, arr->xsum, arr->kty, arr->kty0};
        const double* srcm[6] = {D.y, D.yh, D.y0, D.ysum, D.kx, D.kx0};
        double* dstm[6] = {arr->y, arr->yhat, arr->y0, arr->ysum, arr->kx, arr->kx0};
        std::vector<double> tmp(m);
        for (int k = 0; k < 6; ++k)
            if (dstn[k]) CK(cudaMemcpyAsync(dstn[k], srcn[k], sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int k = 0; k < 6; ++k) {
            if (!dstm[k]) continue;
            CK(cudaMemcpyAsync(tmp.data(), srcm[k], sizeof(double) * m, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int r2 = 0; r2 < m; ++r2) dstm[k][ctx->perm[r2]] = tmp[r2];
        }
        if (arr->soc_root && ctx->n_soc)
            CK(cudaMemcpyAsync(arr->soc_root, ctx->soc_lam, sizeof(float) * ctx->n_soc, cudaMemcpyDeviceToHost, s));
        if (arr->exp_root && ctx->n_exp)
            CK(cudaMemcpyAsync(arr->exp_root, ctx->exp_L, sizeof(float) * ctx->n_exp, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    if (st) {
        const Ctrl& C = *ctx->h_ctrl;
        st->eta = C.eta; st->omega = C.omega; st->wsum = C.wsum; st->phi0 = C.phi0; st->phi_prev = C.phi_prev;
        for (int k = 0; k < 3; ++k) st->comp0[k] = C.comp0[k];
        st->attempts = C.attempts; st->accepted = C.accepted; st->k = C.k; st->restarts = C.restarts;
        st->started = ctx->started ? 1 : 0;
        st->status = C.status;
    }
    return PDCS_OK;
}

pdcs_status pdcs_set_state(pdcs_ctx* ctx, const pdcs_state* st, const pdcs_state_arrays* arr) {
    if (!ctx) return PDCS_ERR_INVALID;
    if (!st || !arr || !arr->x || !arr->x0 || !arr->y || !arr->y0) {
        ctx->err = "pdcs_set_state needs the scalars and x, x0, y, y0";
        return PDCS_ERR_INVALID;
    }
    if (!(st->eta > 0.0) || !(st->omega > 0.0) || !std::isfinite(st->eta) || !std::isfinite(st->omega) ||
        st->status < 0 || st->status > 2 || st->attempts < 0 || st->accepted < 0 || st->k < 0 || st->restarts < 0) {
        ctx->err = "pdcs_set_state: invalid scalars";
        return PDCS_ERR_INVALID;
    }
    const int n = ctx->n, m = ctx->m;
    const double* inn[4] = {arr->x, arr->x0, arr->xsum, nullptr};
    const double* inm[4] = {arr->y, arr->y0, arr->ysum, nullptr};
    for (int k = 0; k < 3; ++k) {
        if (inn[k]) for (int j = 0; j < n; ++j) if (!std::isfinite(inn[k][j])) { ctx->err = "non-finite state"; return PDCS_ERR_INVALID; }
        if (inm[k]) for (int i = 0; i < m; ++i) if (!std::isfinite(inm[k][i])) { ctx->err = "non-finite state"; return PDCS_ERR_INVALID; }
    }
    cudaStream_t s = ctx->stream;
    Dev<double>& D = ctx->D;
    std::vector<double> tmp(m);
    auto put_n = [&](double* dst, const double* h) -> cudaError_t {
        if (!h) return cudaMemsetAsync(dst, 0, sizeof(double) * n, s);
        return cudaMemcpyAsync(dst, h, sizeof(double) * n, cudaMemcpyHostToDevice, s);
    };
    auto put_m = [&](double* dst, const double* h) -> cudaError_t {
        if (!h) return cudaMemsetAsync(dst, 0, sizeof(double) * m, s);
        for (int r = 0; r < m; ++r) tmp[r] = h[ctx->perm[r]];
        cudaError_t e = cudaMemcpyAsync(dst, tmp.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // tmp is reused (pageable)
        return e;
    };
    CK(put_n(D.x, arr->x)); CK(put_n(D.x0, arr->x0)); CK(put_n(D.xsum, arr->xsum));
    CK(put_m(D.y, arr->y)); CK(put_m(D.y0, arr->y0)); CK(put_m(D.ysum, arr->ysum));
    const bool products = arr->kx && arr->kx0 && arr->kty && arr->kty0;
    if (products) {
        CK(put_n(D.kty, arr->kty)); CK(put_n(D.kty0, arr->kty0));
        CK(put_m(D.kx, arr->kx)); CK(put_m(D.kx0, arr->kx0));
    } else {
        launch_spmv<double>(ctx->pk, s, D.rp, D.ci, D.val, D.x, D.kx, nullptr, nullptr, 0, 0);
        launch_spmv<double>(ctx->pk, s, D.rp, D.ci, D.val, D.x0, D.kx0, nullptr, nullptr, 0, 0);
        launch_spmv<double>(ctx->pkt, s, D.rpT, D.ciT, D.valT, D.y, D.kty, nullptr, nullptr, 0, 0);
        launch_spmv<double>(ctx->pkt, s, D.rpT, D.ciT, D.valT, D.y0, D.kty0, nullptr, nullptr, 0, 0);
        ctx->launches += 4;
        CK(cudaGetLastError());
    }
    if (arr->soc_root && ctx->n_soc)
        CK(cudaMemcpyAsync(ctx->soc_lam, arr->soc_root, sizeof(float) * ctx->n_soc, cudaMemcpyHostToDevice, s));
    if (arr->exp_root && ctx->n_exp)
        CK(cudaMemcpyAsync(ctx->exp_L, arr->exp_root, sizeof(float) * ctx->n_exp, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    pdcs_status r = read_ctrl(ctx);
    if (r != PDCS_OK) return r;
    Ctrl C = *ctx->h_ctrl;
    C.eta = st->eta; C.omega = st->omega; C.wsum = st->wsum; C.phi0 = st->phi0; C.phi_prev = st->phi_prev;
    for (int k = 0; k < 3; ++k) C.comp0[k] = st->comp0[k];
    C.attempts = st->attempts; C.accepted = st->accepted; C.k = st->k; C.restarts = st->restarts;
    C.tau = C.eta / C.omega;
    C.sigma = C.eta * C.omega;
    C.pending = 0; C.check_mode = 0; C.restart_now = 0; C.ticket = 0;
    C.xsel = 0; C.xnext = 0;
    C.status = st->status == 0 ? kRunning : (st->status == 1 ? kConverged : kNumericError);
    *ctx->h_ctrl = C;
    CK(cudaMemcpyAsync(ctx->ctrl, ctx->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    ctx->started = st->started != 0;
    ctx->fp32_active = false;
    return PDCS_OK;
}

pdcs_status pdcs_kernel_times(pdcs_ctx* ctx, int64_t attempts, double* ms, int64_t* counts) {
    if (!ctx || !ms || attempts < 1) return PDCS_ERR_INVALID;
    pdcs_status st = read_ctrl(ctx);
    if (st != PDCS_OK) return st;
    if (!ctx->started) {
        const int one = 1;
        CK(cudaMemcpyAsync(&ctx->ctrl->check_mode, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        enqueue_check(ctx);
        ctx->started = true;
    }
    const double zero = 0.0;
    CK(cudaMemcpyAsync(&ctx->ctrl->tol, &zero, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    Prof P;
    long long done = ctx->h_ctrl->attempts;
    for (int64_t a = 0; a < attempts; ++a) {
        enqueue_attempt(ctx, &P);
        ++done;
        if (done % ctx->opt.check_period == 0) enqueue_check(ctx, &P);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < kKernelClasses; ++c) {
        double tot = 0.0;
        const size_t pairs = P.ev[c].size() / 2;
        for (size_t i = 0; i < pairs; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, P.ev[c][2 * i], P.ev[c][2 * i + 1]) == cudaSuccess) tot += t;
        }
        ms[c] = pairs ? tot / (double)pairs : 0.0;
        if (counts) counts[c] = (int64_t)pairs;
        for (cudaEvent_t e : P.ev[c]) cudaEventDestroy(e);
    }
    return read_ctrl(ctx);
}

const char* pdcs_last_error(const pdcs_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void pdcs_destroy(pdcs_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    delete ctx;
}


pdcs_status pdcs_batch_create(pdcs_ctx* const* ctxs, int64_t count, pdcs_batch** out) {
    if (!out) return PDCS_ERR_INVALID;
    *out = nullptr;
    auto bad = [&](const char* m) { g_batch_error = m; return PDCS_ERR_INVALID; };
    if (!ctxs || count < 1 || count > 65535) return bad("count must be in [1, 65535]");
    const pdcs_ctx* c0 = ctxs[0];
    if (!c0) return bad("NULL context");
    for (int64_t i = 0; i < count; ++i) {
        const pdcs_ctx* c = ctxs[i];
        if (!c) return bad("NULL context");
        if (c->opt.batch_blocks <= 0 || c->opt.batch_blocks != c0->opt.batch_blocks)
            return bad("every program needs the same options.batch_blocks > 0");
        if (c->opt.precision != PDCS_PRECISION_FP64) return bad("batches run FP64 programs");
        if (c->opt.check_period != c0->opt.check_period) return bad("programs differ in check_period");
        if (c->pk.unroll != 4 || c->pkt.unroll != 4) return bad("batches use the SpMV unroll 4 (no autotuning)");
        if (c->started) return bad("a program has already been solved alone");
        for (int64_t j = 0; j < i; ++j)
            if (ctxs[j] == c) return bad("a program appears twice");
    }
    pdcs_batch* b = new (std::nothrow) pdcs_batch();
    if (!b) return bad("host allocation failed");
    b->ctxs.assign(ctxs, ctxs + count);
    for (int64_t i = 0; i < count; ++i) b->active.push_back((int)i);
    b->stream = c0->stream;
    b->G = c0->opt.batch_blocks;
    b->period = c0->opt.check_period;
    for (pdcs_ctx* c : b->ctxs)
        b->g_spmv = std::max({b->g_spmv, c->pk.B.blk[c->pk.B.nbins], c->pkt.B.blk[c->pkt.B.nbins], 1});
    std::vector<Dev<double>> hv(count);
    for (int64_t i = 0; i < count; ++i) hv[i] = ctxs[i]->D;
    cudaError_t e = cudaMalloc(&b->views, sizeof(Dev<double>) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMemcpy(b->views, hv.data(), sizeof(Dev<double>) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        g_batch_error = std::string("CUDA: ") + cudaGetErrorString(e);
        delete b;
        return e == cudaErrorMemoryAllocation ? PDCS_ERR_OOM : PDCS_ERR_CUDA;
    }
    *out = b;
    return PDCS_OK;
}

pdcs_status pdcs_batch_solve(pdcs_batch* b, double tol, int64_t max_iter, int64_t* n_converged) {
    if (!b) return PDCS_ERR_INVALID;
    if (max_iter < 0) { b->err = "max_iter < 0"; return PDCS_ERR_INVALID; }
    const double t0 = now_s();
    batch_prepare<<<((int)b->active.size() + 255) / 256, 256, 0, b->stream>>>(b->views, (int)b->active.size(), tol,
                                                                             b->started ? 0 : 1);
    if (!b->started) {
        batch_check(b);  // each program's anchor evaluation
        b->started = true;
        for (pdcs_ctx* c : b->ctxs) c->started = true;
    }
    CKB(cudaGetLastError());
    pdcs_status st = batch_read(b);
    if (st != PDCS_OK) return st;
    long long done = 0;  // all programs advance in lockstep
    {
        Ctrl C;
        CKB(cudaMemcpy(&C, b->ctxs[0]->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
        done = C.attempts;
    }
    long long remaining = max_iter;
    auto running = [&]() {
        for (size_t i = 0; i < b->active.size(); ++i)
            if (b->h_status[i] == kRunning) return true;
        return false;
    };
    while (remaining > 0 && running()) {
        const long long to_b = b->period - (done % b->period);
        if (remaining >= to_b) {
            if (to_b == b->period) {
                if (!b->graph) {
                    cudaGraph_t g;
                    CKB(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                    for (int a = 0; a < b->period; ++a) batch_attempt(b);
                    batch_check(b);
                    CKB(cudaStreamEndCapture(b->stream, &g));
                    cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
                    cudaGraphDestroy(g);
                    if (e != cudaSuccess) { b->graph = nullptr; CKB(e); }
                    // capture only recorded the launches: undo their counts
                    for (int i : b->active)
                        b->ctxs[i]->launches -= (long long)b->period * kLaunchesPerAttempt + kLaunchesPerCheck;
                }
                CKB(cudaGraphLaunch(b->graph, b->stream));
                for (int i : b->active)
                    b->ctxs[i]->launches += (long long)b->period * kLaunchesPerAttempt + kLaunchesPerCheck;
            } else {
                for (long long a = 0; a < to_b; ++a) batch_attempt(b);
                batch_check(b);
            }
            done += to_b;
            remaining -= to_b;
        } else {
            for (long long a = 0; a < remaining; ++a) batch_attempt(b);
            done += remaining;
            remaining = 0;
        }
        CKB(cudaGetLastError());
        st = batch_read(b);
        if (st != PDCS_OK) return st;
        if (done % b->period == 0) {
            st = batch_compact(b);
            if (st != PDCS_OK) return st;
        }
    }
    int conv = 0, numeric = 0;
    const double dt = now_s() - t0;
    for (pdcs_ctx* c : b->ctxs) {
        c->solve_seconds += dt;
        pdcs_status s2 = read_ctrl(c);
        if (s2 != PDCS_OK) return s2;
        c->last_status = status_of(*c->h_ctrl);
        conv += c->h_ctrl->status == kConverged;
        numeric += c->h_ctrl->status == kNumericError;
    }
    const int B = (int)b->ctxs.size();
    if (n_converged) *n_converged = conv;
    if (numeric) { b->err = "NaN or Inf in the iterates of a program"; return PDCS_ERR_NUMERIC; }
    return conv == B ? PDCS_OK : PDCS_MAX_ITER;
}

const char* pdcs_batch_last_error(const pdcs_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

void pdcs_batch_destroy(pdcs_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    delete b;
}

}  // extern "C"
