// wcc_batch_api.cu -- C ABI of batched solving (include/wcc.h, wcc_batch_*):
// many independent 1D problems, one persistent launch per half-step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/wcc.h"
#include "wcc_batch.cuh"
#include "wcc_launch.h"
#include "wcc_trace.h"

using namespace wcc;

namespace {
thread_local std::string g_batch_create_error;
}

struct wcc_batch_ctx {
    int system = 0, nv = 1;
    long long count = 0;
    wcc_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int PA = 0, PB = 0;  // degrees of group 0 / 1 (equal when the batch has one degree)
    int device = 0;      // the device the batch lives on

    std::vector<long long> N;
    std::vector<int> P, bc;
    std::vector<double> dx;
    std::vector<int> order;  // table position -> user index (group 0 first)
    std::vector<BatchInstance> inst;  // table order

    BatchInstance* d_inst = nullptr;
    DevState* d_st = nullptr;
    double* d_hist = nullptr;
    long long hist_cap = 0;
    float* planes[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [group][buffer]
    long long pitch[2] = {0, 0};
    long long* d_tiles_step[2] = {nullptr, nullptr};  // tiles of the launch from a stage of parity s
    long long* d_tiles_cur[2] = {nullptr, nullptr};   // tiles of a stage of parity s
    int* d_inst_step[2] = {nullptr, nullptr};         // instance of every step tile
    int* d_inst_cur[2] = {nullptr, nullptr};          // instance of every auxiliary tile
    long long tiles_step[2] = {0, 0}, tiles_cur[2] = {0, 0};
    long long aos_total[2] = {0, 0};  // doubles of a host-layout stage of parity s
    double* staging = nullptr;
    long long bytes = 0;

    int cur = 0, parity = 0;
    long long steps = 0;
    bool initialised = false;
    int sms = 0, max_ctas_per_sm = 1;
    unsigned grid = 0;  // persistent CTAs of the step kernel

    cudaGraphExec_t gexec = nullptr;
    int g_cur = -1, g_parity = -1, g_chunk = 0;
    double g_cfl = 0.0;
    unsigned g_grid = 0;

    // two half-steps per launch (tb_depth = 2): tiles of kTileTB final cells
    long long* d_tiles_pair[2] = {nullptr, nullptr};
    int* d_inst_pair[2] = {nullptr, nullptr};
    long long tiles_pair[2] = {0, 0};
    DevState* d_backup = nullptr;  // every instance's state before the latest pair launch
    unsigned* d_refused = nullptr; // set when an instance refuses its pair
    double tb_limit[2] = {0.0, 0.0};  // stability limit of each group's degree
    cudaGraphExec_t gexec_tb = nullptr;
    int gt_cur = -1, gt_parity = -1, gt_pairs = 0;
    double gt_cfl = 0.0;
    unsigned gt_grid = 0;
    long long tb_pairs = 0, tb_fallbacks = 0;
    bool pairs_compiled = false;  // the degree mix has a two-half-step kernel

    long long launches = 0;
    std::string err;
};

namespace {

int bfail(wcc_batch_ctx* b, int code, const std::string& msg) {
    if (b) b->err = msg; else g_batch_create_error = msg;
    return code;
}

#define WCC_BCHECK(b, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return bfail((b), WCC_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

long long cells_of(int bc, long long N, int parity) {
    if (bc == WCC_BC_PERIODIC) return N;
    return parity == 0 ? N + 1 : N;
}

long long tiles_of(long long cells) { return (cells + kTile - 1) / kTile; }              // auxiliary kernels
long long step_tiles_of(long long cells) { return (cells + kTileMixed - 1) / kTileMixed; }  // half-step kernel

BatchArgs make_bargs(wcc_batch_ctx* b, int cur, int parity, double cfl, int kind) {
    BatchArgs a{};
    StepArgs& p = a.phys;
    p.limiter = b->opt.limiter;
    p.alpha_is_two = (b->opt.alpha == 2.0);
    p.cfl = cfl;
    p.cfl_mode = 1;
    p.cfl_bits = (unsigned long long)__double_as_longlong_host(cfl);
    p.adv = b->opt.adv_speed;
    p.gamma = b->opt.gamma;
    p.alpha = b->opt.alpha;
    p.eps = b->opt.eps;
    p.gamma_f = (float)b->opt.gamma;
    split_double(b->opt.gamma - 1.0, p.g1_hi, p.g1_lo);
    split_double(b->opt.adv_speed, p.adv_hi, p.adv_lo);
    p.eps_f = (float)b->opt.eps;
    p.alpha_f = (float)b->opt.alpha;
    a.inst = b->d_inst;
    a.st = b->d_st;
    a.hist = b->d_hist;
    a.hist_cap = b->hist_cap;
    for (int g = 0; g < 2; ++g) {
        a.in[g] = b->planes[g][cur];
        a.out[g] = b->planes[g][kind == BATCH_STEP ? cur ^ 1 : cur];
        a.pitch[g] = b->pitch[g];
    }
    if (kind == BATCH_PAIR) {
        for (int g = 0; g < 2; ++g) {
            a.out[g] = b->planes[g][cur ^ 1];
            a.nu_max[g] = std::min(cfl * (1.0 + b->opt.tb_cfl_growth), b->tb_limit[g]);
        }
        a.tile_start = b->d_tiles_pair[parity];
        a.tile_inst = b->d_inst_pair[parity];
        a.total_tiles = b->tiles_pair[parity];
        a.tb_backup = b->d_backup;
        a.tb_refused = b->d_refused;
    } else if (kind == BATCH_STEP) {
        a.tile_start = b->d_tiles_step[parity];
        a.tile_inst = b->d_inst_step[parity];
        a.total_tiles = b->tiles_step[parity];
    } else {
        a.tile_start = b->d_tiles_cur[parity];
        a.tile_inst = b->d_inst_cur[parity];
        a.total_tiles = b->tiles_cur[parity];
    }
    a.ninst = (int)b->count;
    a.parity = parity;
    return a;
}

cudaError_t launch(wcc_batch_ctx* b, int kind, const BatchArgs& a, double* aos, int to_planes, unsigned grid) {
    switch (b->system) {
        case WCC_ADVECTION: return launch_batch<ADVECTION>(b->PA, b->PB, kind, a, aos, to_planes, grid, b->stream);
        case WCC_BURGERS: return launch_batch<BURGERS>(b->PA, b->PB, kind, a, aos, to_planes, grid, b->stream);
        default: return launch_batch<EULER>(b->PA, b->PB, kind, a, aos, to_planes, grid, b->stream);
    }
}

unsigned aux_grid(wcc_batch_ctx* b, long long tiles) {
    long long g = std::min<long long>(tiles, (long long)b->sms * 8);
    return (unsigned)std::max<long long>(g, 1);
}

int read_states(wcc_batch_ctx* b, std::vector<DevState>& st) {
    WCC_BCHECK(b, cudaStreamSynchronize(b->stream));
    st.resize(b->count);
    WCC_BCHECK(b, cudaMemcpy(st.data(), b->d_st, sizeof(DevState) * b->count, cudaMemcpyDeviceToHost));
    unsigned e = 0;
    for (const auto& s : st) e |= s.err;
    if (e & ERR_POSITIVITY) return bfail(b, WCC_E_POSITIVITY, "non-positive density or pressure in an instance");
    if (e & ERR_NONFINITE) return bfail(b, WCC_E_NONFINITE, "a DOF or a CFL bound became NaN/Inf in an instance");
    return WCC_OK;
}

int ensure_hist(wcc_batch_ctx* b, long long need) {
    if (need <= b->hist_cap) return WCC_OK;
    long long cap = b->hist_cap > 0 ? b->hist_cap : 256;
    while (cap < need) cap *= 2;
    double* nh = nullptr;
    WCC_BCHECK(b, cudaStreamSynchronize(b->stream));
    if (cudaMalloc(&nh, (size_t)(cap * b->count) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, WCC_E_NOMEM, "cudaMalloc of the dt histories failed");
    }
    if (b->d_hist) {
        WCC_BCHECK(b, cudaMemcpy2D(nh, cap * sizeof(double), b->d_hist, b->hist_cap * sizeof(double),
                                   b->hist_cap * sizeof(double), b->count, cudaMemcpyDeviceToDevice));
        cudaFree(b->d_hist);
    }
    b->bytes += (cap - b->hist_cap) * b->count * (long long)sizeof(double);
    b->d_hist = nh;
    b->hist_cap = cap;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return WCC_OK;
}

int enqueue_step(wcc_batch_ctx* b, int cur, int parity, double cfl, unsigned grid) {
    BatchArgs a = make_bargs(b, cur, parity, cfl, BATCH_STEP);
    cudaError_t e = launch(b, BATCH_STEP, a, nullptr, 0, grid);
    if (e != cudaSuccess) return bfail(b, WCC_E_CUDA, std::string("batched half-step launch: ") + cudaGetErrorString(e));
    return WCC_OK;
}

int build_graph(wcc_batch_ctx* b, int chunk, double cfl) {
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    WCC_BCHECK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int cur = b->cur, par = b->parity;
    for (int s = 0; s < chunk; ++s) {
        BatchArgs a = make_bargs(b, cur, par, cfl, BATCH_STEP);
        cudaError_t e = launch(b, BATCH_STEP, a, nullptr, 0, b->grid);
        if (e != cudaSuccess) {
            cudaStreamEndCapture(b->stream, &g);
            if (g) cudaGraphDestroy(g);
            return bfail(b, WCC_E_CUDA, std::string("launch during capture: ") + cudaGetErrorString(e));
        }
        cur ^= 1;
        par ^= 1;
    }
    WCC_BCHECK(b, cudaStreamEndCapture(b->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->gexec = nullptr;
        return bfail(b, WCC_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    b->g_cur = b->cur;
    b->g_parity = b->parity;
    b->g_cfl = cfl;
    b->g_chunk = chunk;
    b->g_grid = b->grid;
    return WCC_OK;
}

int enqueue_pair(wcc_batch_ctx* b, int cur, int parity, double cfl, unsigned grid) {
    BatchArgs a = make_bargs(b, cur, parity, cfl, BATCH_PAIR);
    cudaError_t e = launch(b, BATCH_PAIR, a, nullptr, 0, grid);
    if (e != cudaSuccess) return bfail(b, WCC_E_CUDA, std::string("batched two-half-step launch: ") + cudaGetErrorString(e));
    return WCC_OK;
}

// `pairs` (even) two-half-step launches from the current buffer in one graph.
int build_graph_pairs(wcc_batch_ctx* b, int pairs, double cfl) {
    if (b->gexec_tb) {
        cudaGraphExecDestroy(b->gexec_tb);
        b->gexec_tb = nullptr;
    }
    cudaGraph_t g = nullptr;
    WCC_BCHECK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int cur = b->cur;
    for (int s = 0; s < pairs; ++s) {
        BatchArgs a = make_bargs(b, cur, b->parity, cfl, BATCH_PAIR);
        cudaError_t e = launch(b, BATCH_PAIR, a, nullptr, 0, b->grid);
        if (e != cudaSuccess) {
            cudaStreamEndCapture(b->stream, &g);
            if (g) cudaGraphDestroy(g);
            return bfail(b, WCC_E_CUDA, std::string("launch during capture: ") + cudaGetErrorString(e));
        }
        cur ^= 1;
    }
    WCC_BCHECK(b, cudaStreamEndCapture(b->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&b->gexec_tb, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->gexec_tb = nullptr;
        return bfail(b, WCC_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    b->gt_cur = b->cur;
    b->gt_parity = b->parity;
    b->gt_cfl = cfl;
    b->gt_pairs = pairs;
    b->gt_grid = b->grid;
    return WCC_OK;
}

void release(wcc_batch_ctx* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->gexec_tb) cudaGraphExecDestroy(b->gexec_tb);
    for (int s = 0; s < 2; ++s) {
        if (b->d_tiles_pair[s]) cudaFree(b->d_tiles_pair[s]);
        if (b->d_inst_pair[s]) cudaFree(b->d_inst_pair[s]);
    }
    if (b->d_backup) cudaFree(b->d_backup);
    if (b->d_refused) cudaFree(b->d_refused);
    for (int g = 0; g < 2; ++g)
        for (int i = 0; i < 2; ++i)
            if (b->planes[g][i]) cudaFree(b->planes[g][i]);
    for (int s = 0; s < 2; ++s) {
        if (b->d_tiles_step[s]) cudaFree(b->d_tiles_step[s]);
        if (b->d_tiles_cur[s]) cudaFree(b->d_tiles_cur[s]);
        if (b->d_inst_step[s]) cudaFree(b->d_inst_step[s]);
        if (b->d_inst_cur[s]) cudaFree(b->d_inst_cur[s]);
    }
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_st) cudaFree(b->d_st);
    if (b->d_hist) cudaFree(b->d_hist);
    if (b->staging) cudaFree(b->staging);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

int do_step_single(wcc_batch_ctx* b, long long nsteps, double cfl) {
    int rc;
    long long left = nsteps;
    const int chunk = b->opt.graph_chunk;
    if (chunk >= 2 && left >= chunk) {
        if (!b->gexec || b->g_cur != b->cur || b->g_parity != b->parity || b->g_cfl != cfl || b->g_chunk != chunk ||
            b->g_grid != b->grid) {
            rc = build_graph(b, chunk, cfl);
            if (rc != WCC_OK) return rc;
        }
        while (left >= chunk) {
            WCC_BCHECK(b, cudaGraphLaunch(b->gexec, b->stream));
            b->launches += chunk;
            b->steps += chunk;
            left -= chunk;
        }
    }
    for (; left > 0; --left) {
        rc = enqueue_step(b, b->cur, b->parity, cfl, b->grid);
        if (rc != WCC_OK) return rc;
        b->launches += 1;
        b->cur ^= 1;
        b->parity ^= 1;
        b->steps += 1;
    }
    return WCC_OK;
}

// nsteps half-steps as two-half-step launches (an odd last one single),
// checked after the launches: if an instance refused its pair, every
// instance goes back to its state before that launch (the launch left the
// input stages as they were; the launches queued after it did nothing), the
// pair is taken as two single half-steps, and the pairs resume.
int do_step_pairs(wcc_batch_ctx* b, long long nsteps, double cfl) {
    long long pairs = nsteps / 2;
    const int graph_pairs = (b->opt.graph_chunk / 2) & ~1;
    while (pairs > 0) {
        const int cur0 = b->cur;
        const long long steps0 = b->steps;
        long long left = pairs;
        int rc;
        if (graph_pairs >= 2 && left >= graph_pairs) {
            if (!b->gexec_tb || b->gt_cur != b->cur || b->gt_parity != b->parity || b->gt_cfl != cfl ||
                b->gt_pairs != graph_pairs || b->gt_grid != b->grid) {
                if ((rc = build_graph_pairs(b, graph_pairs, cfl)) != WCC_OK) return rc;
            }
            while (left >= graph_pairs) {
                WCC_BCHECK(b, cudaGraphLaunch(b->gexec_tb, b->stream));
                b->launches += graph_pairs;
                b->steps += 2 * graph_pairs;
                left -= graph_pairs;
            }
        }
        for (; left > 0; --left) {
            if ((rc = enqueue_pair(b, b->cur, b->parity, cfl, b->grid)) != WCC_OK) return rc;
            b->launches += 1;
            b->cur ^= 1;
            b->steps += 2;
        }
        unsigned refused = 0;
        WCC_BCHECK(b, cudaMemcpyAsync(&refused, b->d_refused, sizeof refused, cudaMemcpyDeviceToHost, b->stream));
        WCC_BCHECK(b, cudaStreamSynchronize(b->stream));
        if (!refused) {
            b->tb_pairs += pairs;
            break;
        }
        // back to the states before the refused launch, flags cleared
        WCC_BCHECK(b, cudaMemcpyAsync(b->d_st, b->d_backup, sizeof(DevState) * b->count, cudaMemcpyDeviceToDevice,
                                      b->stream));
        WCC_BCHECK(b, cudaMemsetAsync(b->d_refused, 0, sizeof(unsigned), b->stream));
        std::vector<DevState> st;
        if ((rc = read_states(b, st)) != WCC_OK) return rc;
        for (auto& x : st) x.err &= ~ERR_CFL;
        WCC_BCHECK(b, cudaMemcpy(b->d_st, st.data(), sizeof(DevState) * b->count, cudaMemcpyHostToDevice));
        const long long done_pairs = (st[0].step - steps0) / 2;
        b->tb_pairs += done_pairs;
        b->tb_fallbacks += 1;
        b->cur = cur0 ^ (int)(done_pairs & 1);
        b->steps = st[0].step;
        if ((rc = do_step_single(b, 2, cfl)) != WCC_OK) return rc;
        pairs -= done_pairs + 1;
    }
    if (nsteps & 1) return do_step_single(b, 1, cfl);
    return WCC_OK;
}

// cfl above the linear stability limit (Sec. 2.3) of either degree
bool cfl_above_limit(const wcc_batch_ctx* b, double cfl) {
    double la = 0.0, lb = 0.0;
    if (wcc_stability_limit(b->PA, &la) != WCC_OK || wcc_stability_limit(b->PB, &lb) != WCC_OK) return false;
    return cfl > std::min(la, lb);
}

int do_step(wcc_batch_ctx* b, long long nsteps, double cfl) {
    int rc = ensure_hist(b, b->steps + nsteps);
    if (rc != WCC_OK) return rc;
    if (b->opt.tb_depth == 2) return do_step_pairs(b, nsteps, cfl);
    return do_step_single(b, nsteps, cfl);
}

}  // namespace

extern "C" {

int wcc_batch_create(wcc_batch* out, int system, int64_t count, const int64_t* N, const int* P,
                     const double* domains, const int* bcs, const wcc_options* opt) {
    if (!out) return bfail(nullptr, WCC_E_INVAL, "out is NULL");
    *out = nullptr;
    if (system < WCC_ADVECTION || system > WCC_EULER) return bfail(nullptr, WCC_E_INVAL, "unknown system");
    if (count < 1 || count > (1 << 24)) return bfail(nullptr, WCC_E_INVAL, "count must be in 1..2^24");
    if (!N || !P || !domains || !bcs) return bfail(nullptr, WCC_E_INVAL, "NULL array");
    wcc_options o;
    wcc_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != WCC_FP32_MIXED) return bfail(nullptr, WCC_E_INVAL, "batches run in WCC_FP32_MIXED precision");
    if (!(o.eps >= 0.0) || !(o.alpha > 0.0) || !(o.gamma > 1.0) || o.graph_chunk < 0)
        return bfail(nullptr, WCC_E_INVAL, "need eps >= 0, alpha > 0, gamma > 1, graph_chunk >= 0");
    if (o.tb_depth == 0) o.tb_depth = 1;
    if (o.tb_depth != 1 && o.tb_depth != 2) return bfail(nullptr, WCC_E_INVAL, "tb_depth must be 1 or 2");
    if (!(o.tb_cfl_growth >= -1.0) || !(o.tb_cfl_growth < 1e6))
        return bfail(nullptr, WCC_E_INVAL, "tb_cfl_growth must be a number >= -1");
    if (o.cells_per_block != 0 && o.cells_per_block != kTileMixed)
        return bfail(nullptr, WCC_E_INVAL, "batches use tiles of 255 new cells (cells_per_block 0 or 255)");
    int degrees[2] = {0, 0}, nd = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (P[i] < 1 || P[i] > 4) return bfail(nullptr, WCC_E_INVAL, "every P must be in 1..4");
        if (N[i] < 4 || N[i] > (1ll << 31)) return bfail(nullptr, WCC_E_INVAL, "every N must be in 4..2^31");
        if (!(domains[2 * i + 1] > domains[2 * i])) return bfail(nullptr, WCC_E_INVAL, "every domain needs x_L < x_R");
        if (bcs[i] != WCC_BC_PERIODIC && bcs[i] != WCC_BC_TRANSMISSIVE) return bfail(nullptr, WCC_E_INVAL, "unknown bc");
        if (nd == 0 || (P[i] != degrees[0] && (nd < 2 || P[i] != degrees[1]))) {
            if (nd == 2) return bfail(nullptr, WCC_E_INVAL, "a batch holds at most two different degrees P");
            degrees[nd++] = P[i];
        }
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return bfail(nullptr, WCC_E_CUDA, "no CUDA device available");

    wcc_batch_ctx* b = new (std::nothrow) wcc_batch_ctx();
    if (!b) return bfail(nullptr, WCC_E_NOMEM, "host allocation failed");
    b->system = system;
    b->nv = system == WCC_EULER ? 3 : 1;
    b->count = count;
    b->opt = o;
    if (b->opt.graph_chunk & 1) b->opt.graph_chunk += 1;
    if (nd == 1) degrees[1] = degrees[0];
    b->PA = std::min(degrees[0], degrees[1]);
    b->PB = std::max(degrees[0], degrees[1]);
    const int mix = b->PA * 10 + b->PB;
    b->pairs_compiled = mix == 22 || mix == 33 || mix == 23;
    if (o.tb_depth == 2 && !b->pairs_compiled) {
        delete b;
        return bfail(nullptr, WCC_E_INVAL, "two half-steps per launch in a batch: degrees 2 and 3 only");
    }
    if (b->pairs_compiled && (wcc_stability_limit(b->PA, &b->tb_limit[0]) != WCC_OK ||
                              wcc_stability_limit(b->PB, &b->tb_limit[1]) != WCC_OK)) {
        delete b;
        return bfail(nullptr, WCC_E_INVAL, "no stability limit for the batch's degrees");
    }
    b->N.assign(N, N + count);
    b->P.assign(P, P + count);
    b->bc.assign(bcs, bcs + count);
    b->dx.resize(count);
    for (int64_t i = 0; i < count; ++i) b->dx[i] = (domains[2 * i + 1] - domains[2 * i]) / (double)N[i];

    // table order: group 0 (P = PA) then group 1, each in user order
    for (int g = 0; g < 2; ++g)
        for (int64_t i = 0; i < count; ++i)
            if ((g == 0 && P[i] == b->PA) || (g == 1 && P[i] == b->PB && b->PB != b->PA))
                b->order.push_back((int)i);
    // host-layout offsets in user order
    std::vector<long long> aos_off[2];
    for (int s = 0; s < 2; ++s) {
        aos_off[s].resize(count);
        long long acc = 0;
        for (int64_t i = 0; i < count; ++i) {
            aos_off[s][i] = acc;
            acc += cells_of(bcs[i], N[i], s) * b->nv * (P[i] + 1);
        }
        b->aos_total[s] = acc;
    }
    long long goff[2] = {0, 0};
    b->inst.resize(count);
    for (size_t k = 0; k < b->order.size(); ++k) {
        const int i = b->order[k];
        BatchInstance& I = b->inst[k];
        I.group = (P[i] == b->PA) ? 0 : 1;
        I.offset = goff[I.group];
        goff[I.group] += (cells_of(bcs[i], N[i], 0) + 31) / 32 * 32;  // 128-byte aligned instances
        I.aos_offset[0] = aos_off[0][i];
        I.aos_offset[1] = aos_off[1][i];
        I.cells[0] = cells_of(bcs[i], N[i], 0);
        I.cells[1] = cells_of(bcs[i], N[i], 1);
        I.dx = b->dx[i];
        I.bc = bcs[i];
    }
    std::vector<long long> ts[2], tc[2];
    for (int s = 0; s < 2; ++s) {
        ts[s].assign(count + 1, 0);
        tc[s].assign(count + 1, 0);
        for (int64_t k = 0; k < count; ++k) {
            ts[s][k + 1] = ts[s][k] + step_tiles_of(b->inst[k].cells[s ^ 1]);
            tc[s][k + 1] = tc[s][k] + tiles_of(b->inst[k].cells[s]);
        }
        b->tiles_step[s] = ts[s][count];
        b->tiles_cur[s] = tc[s][count];
    }
    // pair tiles: kTileTB final cells of the stage of the same parity
    std::vector<long long> tp[2];
    for (int s = 0; s < 2; ++s) {
        tp[s].assign(count + 1, 0);
        for (int64_t k = 0; k < count; ++k)
            tp[s][k + 1] = tp[s][k] + (b->inst[k].cells[s] + kTileTB - 1) / kTileTB;
        b->tiles_pair[s] = tp[s][count];
    }

    if (o.cuda_stream) {
        b->stream = (cudaStream_t)o.cuda_stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
        b->own_stream = true;
    } else {
        delete b;
        return bfail(nullptr, WCC_E_CUDA, "cudaStreamCreate failed");
    }
    int dev = 0;
    cudaGetDevice(&dev);
    b->device = dev;
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);

    bool ok = true;
    auto dmalloc = [&](void** p, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            return;
        }
        b->bytes += (long long)bytes;
    };
    for (int g = 0; g < 2; ++g) {
        b->pitch[g] = std::max<long long>((goff[g] + 63) / 64 * 64, 64);
        if (g == 1 && b->PB == b->PA) continue;
        const int P_g = g == 0 ? b->PA : b->PB;
        const size_t bytes = (size_t)(b->nv * (P_g + 2) * b->pitch[g]) * sizeof(float);
        for (int i = 0; i < 2; ++i) {
            dmalloc((void**)&b->planes[g][i], bytes);
            if (ok) cudaMemsetAsync(b->planes[g][i], 0, bytes, b->stream);
        }
    }
    if (b->PB == b->PA) {  // group 1 is empty: alias group 0 so that no pointer is NULL
        b->planes[1][0] = nullptr;
        b->planes[1][1] = nullptr;
    }
    dmalloc((void**)&b->d_inst, sizeof(BatchInstance) * count);
    dmalloc((void**)&b->d_st, sizeof(DevState) * count);
    std::vector<int> is[2], ic[2];
    for (int s = 0; s < 2; ++s) {
        dmalloc((void**)&b->d_tiles_step[s], sizeof(long long) * (count + 1));
        dmalloc((void**)&b->d_tiles_cur[s], sizeof(long long) * (count + 1));
        is[s].resize(b->tiles_step[s]);
        ic[s].resize(b->tiles_cur[s]);
        for (int64_t k = 0; k < count; ++k) {
            for (long long t = ts[s][k]; t < ts[s][k + 1]; ++t) is[s][t] = (int)k;
            for (long long t = tc[s][k]; t < tc[s][k + 1]; ++t) ic[s][t] = (int)k;
        }
        dmalloc((void**)&b->d_inst_step[s], sizeof(int) * std::max<long long>(b->tiles_step[s], 1));
        dmalloc((void**)&b->d_inst_cur[s], sizeof(int) * std::max<long long>(b->tiles_cur[s], 1));
    }
    std::vector<int> ip[2];
    if (b->pairs_compiled) {
        for (int s = 0; s < 2; ++s) {
            dmalloc((void**)&b->d_tiles_pair[s], sizeof(long long) * (count + 1));
            ip[s].resize(b->tiles_pair[s]);
            for (int64_t k = 0; k < count; ++k)
                for (long long t = tp[s][k]; t < tp[s][k + 1]; ++t) ip[s][t] = (int)k;
            dmalloc((void**)&b->d_inst_pair[s], sizeof(int) * std::max<long long>(b->tiles_pair[s], 1));
        }
        dmalloc((void**)&b->d_backup, sizeof(DevState) * count);
        dmalloc((void**)&b->d_refused, sizeof(unsigned));
    }
    dmalloc((void**)&b->staging, sizeof(double) * (size_t)std::max(b->aos_total[0], b->aos_total[1]));
    if (!ok) {
        release(b);
        delete b;
        return bfail(nullptr, WCC_E_NOMEM, "cudaMalloc of the batch state failed");
    }
    cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(BatchInstance) * count, cudaMemcpyHostToDevice, b->stream);
    for (int s = 0; s < 2; ++s) {
        cudaMemcpyAsync(b->d_tiles_step[s], ts[s].data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(b->d_tiles_cur[s], tc[s].data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(b->d_inst_step[s], is[s].data(), sizeof(int) * is[s].size(), cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(b->d_inst_cur[s], ic[s].data(), sizeof(int) * ic[s].size(), cudaMemcpyHostToDevice, b->stream);
    }
    if (b->pairs_compiled) {
        for (int s = 0; s < 2; ++s) {
            cudaMemcpyAsync(b->d_tiles_pair[s], tp[s].data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice,
                            b->stream);
            cudaMemcpyAsync(b->d_inst_pair[s], ip[s].data(), sizeof(int) * ip[s].size(), cudaMemcpyHostToDevice,
                            b->stream);
        }
        cudaMemsetAsync(b->d_refused, 0, sizeof(unsigned), b->stream);
    }
    cudaStreamSynchronize(b->stream);  // the host vectors go out of scope
    cudaMemsetAsync(b->d_st, 0, sizeof(DevState) * count, b->stream);
    switch (system) {
        case WCC_ADVECTION: b->max_ctas_per_sm = batch_blocks_per_sm<ADVECTION>(b->PA, b->PB); break;
        case WCC_BURGERS: b->max_ctas_per_sm = batch_blocks_per_sm<BURGERS>(b->PA, b->PB); break;
        default: b->max_ctas_per_sm = batch_blocks_per_sm<EULER>(b->PA, b->PB); break;
    }
    if (b->max_ctas_per_sm < 1) b->max_ctas_per_sm = 1;
    b->grid = (unsigned)(b->max_ctas_per_sm * b->sms);
    if (ensure_hist(b, 1024) != WCC_OK || cudaStreamSynchronize(b->stream) != cudaSuccess) {
        std::string m = b->err;
        release(b);
        delete b;
        return bfail(nullptr, WCC_E_CUDA, "batch set-up failed: " + m);
    }
    *out = b;
    return WCC_OK;
}

int wcc_batch_dof_count(wcc_batch b, int64_t* count) {
    if (!b || !count) return bfail(b, WCC_E_INVAL, "NULL argument");
    *count = b->aos_total[b->parity];
    return WCC_OK;
}

int wcc_batch_set_initial(wcc_batch b, const double* dofs, int64_t count) {
    WccTraceRange trace_("wcc_batch_set_initial");
    if (!b) return bfail(nullptr, WCC_E_INVAL, "NULL batch");
    DeviceScope ds_(b->device);
    if (!dofs) return bfail(b, WCC_E_INVAL, "dofs is NULL");
    if (count != b->aos_total[0]) return bfail(b, WCC_E_INVAL, "count does not match the integer stages of the batch");
    WCC_BCHECK(b, cudaMemcpyAsync(b->staging, dofs, (size_t)count * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    b->cur = 0;
    b->parity = 0;
    b->steps = 0;
    b->tb_pairs = b->tb_fallbacks = 0;
    BatchArgs a = make_bargs(b, 0, 0, 1.0, BATCH_CONVERT);
    cudaError_t e = launch(b, BATCH_CONVERT, a, b->staging, 1, aux_grid(b, a.total_tiles));
    if (e != cudaSuccess) return bfail(b, WCC_E_CUDA, std::string("layout conversion: ") + cudaGetErrorString(e));
    WCC_BCHECK(b, cudaMemsetAsync(b->d_st, 0, sizeof(DevState) * b->count, b->stream));
    a = make_bargs(b, 0, 0, 1.0, BATCH_SPEED);
    e = launch(b, BATCH_SPEED, a, nullptr, 0, aux_grid(b, a.total_tiles));
    if (e != cudaSuccess) return bfail(b, WCC_E_CUDA, std::string("stage bound: ") + cudaGetErrorString(e));
    b->launches += 2;
    b->initialised = true;
    std::vector<DevState> st;
    int rc = read_states(b, st);
    if (rc != WCC_OK) b->initialised = false;
    return rc;
}

int wcc_batch_step(wcc_batch b, int64_t nsteps, double cfl) {
    WccTraceRange trace_("wcc_batch_step");
    if (!b) return bfail(nullptr, WCC_E_INVAL, "NULL batch");
    DeviceScope ds_(b->device);
    if (!b->initialised) return bfail(b, WCC_E_STATE, "wcc_batch_set_initial has not been called");
    if (nsteps < 0 || !(cfl > 0.0) || !(cfl < 1e6)) return bfail(b, WCC_E_INVAL, "need nsteps >= 0 and cfl > 0");
    if (cfl_above_limit(b, cfl))
        return bfail(b, WCC_E_CFL, "cfl above the linear stability limit of a degree (wcc_stability_limit)");
    return do_step(b, nsteps, cfl);
}

int wcc_batch_get_dofs(wcc_batch b, double* dofs, int64_t count) {
    WccTraceRange trace_("wcc_batch_get_dofs");
    if (!b) return bfail(nullptr, WCC_E_INVAL, "NULL batch");
    DeviceScope ds_(b->device);
    if (!dofs) return bfail(b, WCC_E_INVAL, "dofs is NULL");
    if (!b->initialised) return bfail(b, WCC_E_STATE, "wcc_batch_set_initial has not been called");
    if (count != b->aos_total[b->parity]) return bfail(b, WCC_E_INVAL, "count does not match the current stages");
    BatchArgs a = make_bargs(b, b->cur, b->parity, 1.0, BATCH_CONVERT);
    cudaError_t e = launch(b, BATCH_CONVERT, a, b->staging, 0, aux_grid(b, a.total_tiles));
    if (e != cudaSuccess) return bfail(b, WCC_E_CUDA, std::string("layout conversion: ") + cudaGetErrorString(e));
    b->launches += 1;
    WCC_BCHECK(b, cudaMemcpyAsync(dofs, b->staging, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    std::vector<DevState> st;
    return read_states(b, st);
}

int wcc_batch_get_times(wcc_batch b, double* t, int64_t count) {
    if (!b || !t || count != b->count) return bfail(b, WCC_E_INVAL, "need t[count] with count = instances");
    DeviceScope ds_(b->device);
    std::vector<DevState> st;
    int rc = read_states(b, st);
    for (size_t k = 0; k < b->order.size(); ++k) t[b->order[k]] = st[k].t;
    return rc;
}

int wcc_batch_get_state(wcc_batch b, int64_t* half_steps, int* parity) {
    if (!b) return bfail(nullptr, WCC_E_INVAL, "NULL batch");
    DeviceScope ds_(b->device);
    std::vector<DevState> st;
    int rc = read_states(b, st);
    if (half_steps) *half_steps = b->steps;
    if (parity) *parity = b->parity;
    return rc;
}

int wcc_batch_get_dt_history(wcc_batch b, int64_t instance, double* dts, int64_t cap, int64_t* n) {
    if (!b) return bfail(nullptr, WCC_E_INVAL, "NULL batch");
    DeviceScope ds_(b->device);
    if (instance < 0 || instance >= b->count || cap < 0 || (cap > 0 && !dts))
        return bfail(b, WCC_E_INVAL, "bad instance / dts / cap");
    std::vector<DevState> st;
    int rc = read_states(b, st);
    const long long k = std::find(b->order.begin(), b->order.end(), (int)instance) - b->order.begin();
    const long long taken = st[k].step;
    if (n) *n = taken;
    long long m = std::min<long long>(std::min<long long>(taken, cap), b->hist_cap);
    if (m > 0)
        WCC_BCHECK(b, cudaMemcpy(dts, b->d_hist + k * b->hist_cap, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost));
    return rc;
}

int wcc_batch_tb_stats(wcc_batch b, int64_t* pairs, int64_t* fallbacks) {
    if (!b) return bfail(nullptr, WCC_E_INVAL, "NULL batch");
    DeviceScope ds_(b->device);
    std::vector<DevState> st;
    int rc = read_states(b, st);
    if (pairs) *pairs = b->tb_pairs;
    if (fallbacks) *fallbacks = b->tb_fallbacks;
    return rc;
}

int wcc_batch_set_grid(wcc_batch b, int ctas) {
    if (!b) return bfail(nullptr, WCC_E_INVAL, "NULL batch");
    DeviceScope ds_(b->device);
    if (ctas < 0) return bfail(b, WCC_E_INVAL, "ctas must be >= 0");
    b->grid = ctas == 0 ? (unsigned)(b->max_ctas_per_sm * b->sms) : (unsigned)ctas;
    return WCC_OK;
}

int wcc_batch_autotune(wcc_batch b, double cfl, int* ctas_out) {
    if (!b) return bfail(nullptr, WCC_E_INVAL, "NULL batch");
    DeviceScope ds_(b->device);
    if (!b->initialised) return bfail(b, WCC_E_STATE, "wcc_batch_set_initial has not been called");
    if (!(cfl > 0.0)) return bfail(b, WCC_E_INVAL, "cfl must be positive");
    if (cfl_above_limit(b, cfl))
        return bfail(b, WCC_E_CFL, "cfl above the linear stability limit of a degree (wcc_stability_limit)");
    // Candidates: persistent grids of 1..max resident CTAs per SM and one
    // CTA per tile, each with one half-step per launch and (where the degree
    // mix has the kernel) two.  Each is timed over eight half-steps on the
    // batch itself; the state is restored afterwards.
    struct Cand {
        unsigned grid;
        int tb;
    };
    std::vector<Cand> cand;
    for (int tb = 1; tb <= (b->pairs_compiled ? 2 : 1); ++tb) {
        for (int k = 1; k <= b->max_ctas_per_sm; ++k) cand.push_back({(unsigned)(k * b->sms), tb});
        const long long tiles = tb == 1 ? std::max(b->tiles_step[0], b->tiles_step[1])
                                        : std::max(b->tiles_pair[0], b->tiles_pair[1]);
        cand.push_back({(unsigned)std::min<long long>(tiles, 1ll << 30), tb});
    }
    const int G = b->PB == b->PA ? 1 : 2;
    size_t plane_bytes[2] = {0, 0};
    for (int g = 0; g < G; ++g)
        plane_bytes[g] = (size_t)(b->nv * ((g == 0 ? b->PA : b->PB) + 2) * b->pitch[g]) * sizeof(float);
    void* save = nullptr;
    const size_t save_bytes = plane_bytes[0] + plane_bytes[1] + sizeof(DevState) * b->count;
    if (cudaMalloc(&save, save_bytes) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, WCC_E_NOMEM, "autotune: cudaMalloc of the state copy failed");
    }
    char* sp = (char*)save;
    const int cur0 = b->cur, par0 = b->parity;
    const long long steps0 = b->steps;
    auto restore_copy = [&](bool to_save) {
        size_t off = 0;
        for (int g = 0; g < G; ++g) {
            if (to_save) cudaMemcpyAsync(sp + off, b->planes[g][cur0], plane_bytes[g], cudaMemcpyDeviceToDevice, b->stream);
            else cudaMemcpyAsync(b->planes[g][cur0], sp + off, plane_bytes[g], cudaMemcpyDeviceToDevice, b->stream);
            off += plane_bytes[g];
        }
        if (to_save) cudaMemcpyAsync(sp + off, b->d_st, sizeof(DevState) * b->count, cudaMemcpyDeviceToDevice, b->stream);
        else cudaMemcpyAsync(b->d_st, sp + off, sizeof(DevState) * b->count, cudaMemcpyDeviceToDevice, b->stream);
        if (!to_save && b->d_refused) cudaMemsetAsync(b->d_refused, 0, sizeof(unsigned), b->stream);
    };
    int rc = ensure_hist(b, steps0 + 16);
    if (rc != WCC_OK) {
        cudaFree(save);
        return rc;
    }
    restore_copy(true);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    unsigned best_grid = b->grid;
    int best_tb = b->opt.tb_depth;
    for (const Cand& c : cand) {
        const unsigned grid = c.grid;
        int cur = cur0, par = par0;
        if (c.tb == 1) {
            for (int s = 0; s < 10 && rc == WCC_OK; ++s) {
                if (s == 2) cudaEventRecord(e0, b->stream);
                rc = enqueue_step(b, cur, par, cfl, grid);
                cur ^= 1;
                par ^= 1;
            }
        } else {
            cudaMemsetAsync(b->d_refused, 0, sizeof(unsigned), b->stream);
            for (int s = 0; s < 5 && rc == WCC_OK; ++s) {
                if (s == 1) cudaEventRecord(e0, b->stream);
                rc = enqueue_pair(b, cur, par, cfl, grid);
                cur ^= 1;
            }
        }
        cudaEventRecord(e1, b->stream);
        if (rc != WCC_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = rc != WCC_OK ? rc : WCC_E_CUDA;
            restore_copy(false);  // the stage as it was, as far as the context allows
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        // A refused pair leaves the launches after it with nothing to do, so
        // the time says nothing; the state also made this batch refuse a
        // pair, and the depth that needs no redoing is kept.
        unsigned refused = 0;
        if (c.tb == 2 && (cudaMemcpyAsync(&refused, b->d_refused, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream) !=
                              cudaSuccess ||
                          cudaStreamSynchronize(b->stream) != cudaSuccess)) {
            rc = WCC_E_CUDA;
            restore_copy(false);
            break;
        }
        if (!refused && ms < best) {
            best = ms;
            best_grid = grid;
            best_tb = c.tb;
        }
        restore_copy(false);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(b->stream);
    cudaFree(save);
    if (rc != WCC_OK) return rc;
    b->grid = best_grid;
    b->opt.tb_depth = best_tb;
    b->cur = cur0;
    b->parity = par0;
    b->steps = steps0;
    if (ctas_out) *ctas_out = (int)best_grid;
    return WCC_OK;
}

int wcc_batch_get_tuning(wcc_batch b, int* ctas, int* tb_depth) {
    if (!b) return bfail(nullptr, WCC_E_INVAL, "NULL batch");
    if (ctas) *ctas = (int)b->grid;
    if (tb_depth) *tb_depth = b->opt.tb_depth;
    return WCC_OK;
}

int wcc_batch_synchronize(wcc_batch b) {
    if (!b) return bfail(nullptr, WCC_E_INVAL, "NULL batch");
    DeviceScope ds_(b->device);
    std::vector<DevState> st;
    return read_states(b, st);
}

int wcc_batch_launch_count(wcc_batch b, int64_t* launches) {
    if (!b || !launches) return bfail(b, WCC_E_INVAL, "NULL argument");
    *launches = b->launches;
    return WCC_OK;
}

int wcc_batch_device_bytes(wcc_batch b, int64_t* bytes) {
    if (!b || !bytes) return bfail(b, WCC_E_INVAL, "NULL argument");
    *bytes = b->bytes;
    return WCC_OK;
}

const char* wcc_batch_last_error(wcc_batch b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

void wcc_batch_destroy(wcc_batch b) {
    if (!b) return;
    DeviceScope ds_(b->device);
    cudaStreamSynchronize(b->stream);
    release(b);
    delete b;
}

}  // extern "C"
