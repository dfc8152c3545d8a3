// server.cu -- serving: continuous batching of independent fits of one model kind (paper
// Sec. 2.1 fits, run many at a time).  A server owns fixed fit slots and a device event pool
// (the HBM budget); a request is admitted into a free slot when the pool has room for its
// events, every step advances all busy slots by one device step of the batched fit loop
// (batch.cu: prepare, evaluate, update, replayed from a CUDA graph), and finished fits are
// collected, freeing their slot and pool range for the next admissions.  Each fit's sums are
// reduced in its own fixed order, so a result does not depend on which fits share the steps.
//
// Two streams keep the device busy while the host admits and collects:
//   step stream        the graph steps, and the analytic start-matrix pass of newly admitted
//                      fits (strategy 2) queued ahead of the next step;
//   collection stream  admission (the copy of a request's events into its free pool range,
//                      the range check, sum (m - ma), the angular basis) and collection (Newton
//                      polish with the analytic Hessian, hessian 2 / 3, and the packing of the
//                      results of finished fits).
// Admission writes only a free pool range and installs the new fit state on the step stream
// (from pinned staging, behind the steps already queued); collection touches only fits that
// have finished, which the steps skip (the update kernel publishes a fit's final state, then
// its done flag in mapped memory), so neither waits for the steps in flight.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/gbnll.h"
#include "batch_internal.h"
#include "trace.h"
#include "gbnll_internal.h"

using namespace gbnll;

namespace {
const double kPiH = 3.14159265358979323846;
constexpr int kStepRing = 64;  // events of the most recent graph steps (steps in flight)
}  // namespace

struct nll_server {
    int kind = 0, ndim = 0, npar = 0, device = 0, sm_count = 0;
    DevBudget budget;  // device memory of this server (limit from GBNLL_DEVICE_ALLOC_LIMIT)
    cudaStream_t stream = nullptr;   // steps and start passes
    cudaStream_t cstream = nullptr;  // admission and collection (highest stream priority)
    double ranges[8] = {0};
    int max_slots = 0;
    int64_t pool_events = 0, n_pad = 0;
    int ncols = 0, tile_events = 4096;
    double* d_ev = nullptr;
    std::vector<std::pair<int64_t, int64_t>> free_ranges;  // [begin, end) in pool events, sorted
    std::vector<char> busy;
    std::vector<int64_t> slot_id, slot_begin, slot_len, slot_nev;
    std::vector<int> need_start;  // strategy 2: admitted slots whose start matrix is still due
    int64_t next_id = 1;
    FitConfig cfg;
    int hessian = 0;  // fit_options.hessian: 2 / 3 polish finished slots with the analytic Hessian
    bool subsample_start = false;  // strategy 3: start matrices from a subsample of each fit's events
    bool single_start = false;     // strategy 5: start matrices from a single-precision event pass
    HessWork hw;      // start passes (strategy 2), on the step stream
    HessWork hwp;     // polish passes (hessian 2 / 3), on the collection stream
    // admission statistics on the device (range check, sum (m - ma)) of a request's events
    double* d_spart = nullptr;
    unsigned int* d_sticket = nullptr;
    double* h_sout = nullptr;  // mapped [3]
    double* d_sout = nullptr;
    std::vector<double> step;
    // pinned staging of admitted fit states (installed by copies on the step stream)
    ToyFit* h_fit_stage = nullptr;
    int64_t* h_be_stage = nullptr;  // [slot][2]: begin, end
    double* h_sum_stage = nullptr;  // [slot]
    // collection: slot list (pinned and device) and packed results (mapped)
    int* h_pick = nullptr;
    int* d_pick = nullptr;
    double* h_res = nullptr;
    double* d_res = nullptr;
    // device work arrays
    int64_t* d_begin = nullptr;
    int64_t* d_end = nullptr;
    double* d_sum_wdm = nullptr;
    ToyFit* d_fits = nullptr;
    int* d_counters = nullptr;
    int* h_active = nullptr;
    int* d_active = nullptr;
    int* h_done = nullptr;
    int* d_done = nullptr;
    int* d_item_toy = nullptr;
    int* d_item_u0 = nullptr;
    int* d_item_nt = nullptr;
    KConst* d_item_kc = nullptr;
    DConst* d_item_dc = nullptr;
    int* d_unit_item = nullptr;
    int* d_unit_tile = nullptr;
    double* d_unit_sums = nullptr;
    int max_items = 0, max_units = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // events of the last kStepRing graph steps: steps in flight without a stream query
    cudaEvent_t step_ev[kStepRing] = {};
    int step_head = 0;
    std::string err;
};

namespace {

int sfail(nll_server* s, int status, const char* fmt, ...)
{
    if (s) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        s->err = buf;
    }
    return status;
}

void server_free(nll_server* s)
{
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    void* ptrs[] = {s->d_ev, s->d_begin, s->d_end, s->d_sum_wdm, s->d_fits, s->d_counters, s->d_item_toy,
                    s->d_item_u0, s->d_item_nt, s->d_item_kc, s->d_item_dc, s->d_unit_item, s->d_unit_tile,
                    s->d_unit_sums, s->d_spart, s->d_sticket, s->d_pick};
    for (void* p : ptrs)
        if (p) gb_free(p);
    void* hptrs[] = {s->h_active, s->h_done, s->h_sout, s->h_fit_stage, s->h_be_stage, s->h_sum_stage, s->h_pick,
                     s->h_res};
    for (void* p : hptrs)
        if (p) cudaFreeHost(p);
    hw_free(s->hw);
    hw_free(s->hwp);
    for (auto& ev : s->step_ev)
        if (ev) cudaEventDestroy(ev);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->cstream) cudaStreamDestroy(s->cstream);
}

// first-fit allocation of `len` (even) pool events starting on an even event
bool pool_alloc(nll_server* s, int64_t len, int64_t* begin)
{
    for (size_t i = 0; i < s->free_ranges.size(); ++i) {
        auto& r = s->free_ranges[i];
        if (r.second - r.first >= len) {
            *begin = r.first;
            r.first += len;
            if (r.first == r.second) s->free_ranges.erase(s->free_ranges.begin() + i);
            return true;
        }
    }
    return false;
}

void pool_release(nll_server* s, int64_t begin, int64_t len)
{
    auto& fr = s->free_ranges;
    auto it = std::lower_bound(fr.begin(), fr.end(), std::make_pair(begin, begin + len));
    it = fr.insert(it, {begin, begin + len});
    // merge with neighbours
    size_t i = it - fr.begin();
    if (i + 1 < fr.size() && fr[i].second == fr[i + 1].first) {
        fr[i].second = fr[i + 1].second;
        fr.erase(fr.begin() + i + 1);
    }
    if (i > 0 && fr[i - 1].second == fr[i].first) {
        fr[i - 1].second = fr[i].second;
        fr.erase(fr.begin() + i);
    }
}

BatchDev server_dev(nll_server* s)
{
    BatchDev d;
    memset(&d, 0, sizeof d);
    d.n_toys = s->max_slots;
    d.tile_pairs = s->tile_events / 2;
    d.ev_begin = s->d_begin;
    d.ev_end = s->d_end;
    d.sum_wdm = s->d_sum_wdm;
    for (int c = 0; c < kNumCols; ++c) d.cols.col[c] = c < s->ncols ? s->d_ev + (size_t)c * s->n_pad : nullptr;
    d.cols.w = nullptr;
    d.fits = s->d_fits;
    d.counters = s->d_counters;
    d.n_active = s->d_active;
    d.done_flags = s->d_done;
    d.item_toy = s->d_item_toy;
    d.item_u0 = s->d_item_u0;
    d.item_nt = s->d_item_nt;
    d.item_kc = s->d_item_kc;
    d.item_dc = s->d_item_dc;
    d.unit_item = s->d_unit_item;
    d.unit_tile = s->d_unit_tile;
    d.unit_sums = s->d_unit_sums;
    d.max_items = s->max_items;
    d.max_units = s->max_units;
    d.cfg = s->cfg;
    return d;
}

HessTarget server_target(nll_server* s, cudaStream_t stream)
{
    HessTarget T;
    memset(&T, 0, sizeof T);
    T.kind = s->kind;
    T.variant = kVarPrecompute;  // the server builds the angular basis at admission
    T.sm_count = s->sm_count;
    T.n_toys = s->max_slots;
    T.weighted = false;
    for (int c = 0; c < kNumCols; ++c) T.ev.col[c] = c < s->ncols ? s->d_ev + (size_t)c * s->n_pad : nullptr;
    T.d_begin = s->d_begin;
    T.d_end = s->d_end;
    T.d_sum_wdm = s->d_sum_wdm;
    T.d_fits = s->d_fits;
    T.stream = stream;
    return T;
}

// unit lists of a Hessian pass over the slots with pick[i] != 0
cudaError_t server_pick(nll_server* s, HessWork& w, const std::vector<int>& pick, cudaStream_t stream, bool wait,
                        bool subsample = false)
{
    std::vector<int64_t> begin(s->max_slots), end(s->max_slots);
    for (int i = 0; i < s->max_slots; ++i) {
        begin[i] = s->slot_begin[i];
        end[i] = s->slot_begin[i] + (pick[i] ? s->slot_nev[i] : 0);
    }
    return hw_set_units(w, begin, end, pick, stream, wait, subsample);
}

int finished_count(const nll_server* s)
{
    int n = 0;
    for (int i = 0; i < s->max_slots; ++i)
        if (s->busy[i] && ((volatile const int*)s->h_done)[i]) ++n;
    return n;
}

}  // namespace

extern "C" {

int nll_server_create(int kind, const double* obs_ranges, int device, int max_slots, int64_t pool_events,
                      int tile_events, const double* lo, const double* hi, const double* step, const int* fixed,
                      const fit_options* opt_in, nll_server** out)
{
    if (!out) return NLL_ERR_ARG;
    *out = nullptr;
    if (opt_in && (opt_in->strategy < 0 || opt_in->strategy > 5 || opt_in->strategy == 4 || opt_in->hessian < 0 ||
                   opt_in->hessian > 3))
        return NLL_ERR_ARG;
    if ((kind != NLL_MODEL_MASS1D && kind != NLL_MODEL_KSTARMUMU4D) || !obs_ranges || max_slots < 1 ||
        pool_events < 1 || tile_events < 0 || (tile_events > 0 && (tile_events < 128 || (tile_events & 1))))
        return NLL_ERR_ARG;
    if (!(isfinite(obs_ranges[0]) && isfinite(obs_ranges[1]) && obs_ranges[0] < obs_ranges[1])) return NLL_ERR_ARG;
    if (kind == NLL_MODEL_KSTARMUMU4D) {
        const double want[6] = {-1.0, 1.0, -1.0, 1.0, -kPiH, kPiH};
        for (int i = 0; i < 6; ++i)
            if (fabs(obs_ranges[2 + i] - want[i]) > 1e-12) return NLL_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return NLL_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return NLL_ERR_CUDA;
    nll_server* s = new nll_server();
    s->budget.limit = dev_budget_limit_from_env();
    s->hw.budget = &s->budget;
    s->hwp.budget = &s->budget;
    s->kind = kind;
    s->ndim = kind == NLL_MODEL_MASS1D ? 1 : 4;
    s->npar = kind == NLL_MODEL_MASS1D ? 4 : 18;
    s->device = device;
    s->max_slots = max_slots;
    s->tile_events = tile_events ? tile_events : 4096;
    memcpy(s->ranges, obs_ranges, sizeof(double) * 2 * s->ndim);
    if (kind == NLL_MODEL_KSTARMUMU4D) {
        s->ranges[6] = -kPiH;
        s->ranges[7] = kPiH;
    }
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, device);
    fit_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        memset(&opt, 0, sizeof opt);
    if (!(opt.tol_edm > 0.0)) opt.tol_edm = 1e-8;
    if (opt.max_iter <= 0) opt.max_iter = 500;
    memset(&s->cfg, 0, sizeof s->cfg);
    s->cfg.kind = kind;
    s->cfg.npar = s->npar;
    for (int i = 0; i < 8; ++i) s->cfg.ranges[i] = s->ranges[i];
    setup_config(s->cfg, s->npar, lo, hi, step, fixed, opt);
    s->hessian = opt.hessian;
    s->subsample_start = opt.strategy == 3;
    s->single_start = opt.strategy == 5;
    s->step.assign(s->npar, 0.0);
    for (int k = 0; k < s->npar; ++k) s->step[k] = step ? step[k] : 0.0;
    // pool: padded so a range of even length starting on an even event can end anywhere
    s->pool_events = (pool_events + 1) & ~int64_t(1);
    s->n_pad = std::max<int64_t>((s->pool_events + 63) / 64 * 64, 64);
    s->ncols = kind == kMass1D ? 1 : kNumCols;
    s->free_ranges.push_back({0, s->pool_events});
    s->busy.assign(max_slots, 0);
    s->slot_id.assign(max_slots, 0);
    s->slot_begin.assign(max_slots, 0);
    s->slot_len.assign(max_slots, 0);
    s->slot_nev.assign(max_slots, 0);
    s->need_start.assign(max_slots, 0);
    const int64_t tp = s->tile_events / 2;
    s->max_items = max_slots * (2 * s->npar + 1);
    int64_t mu = (s->pool_events / 2 / tp + max_slots + 1) * (2 * (int64_t)s->npar + 1);
    if (mu > (1ll << 30)) {
        delete s;
        return NLL_ERR_ARG;
    }
    s->max_units = (int)mu;
    cudaError_t e = ensure_btab(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    // admissions and collections wait on the host: their kernels go ahead of queued step blocks
    int prio_least = 0, prio_greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->cstream, cudaStreamNonBlocking, prio_greatest);
    // every slot's Hessian units fit: the pool holds at most pool_events events
    const int64_t cap = s->pool_events / kHessUnitEvents + max_slots + 1;
    if (e == cudaSuccess && s->cfg.strategy == 2)
        e = cap > (1 << 28) ? cudaErrorInvalidValue : hw_alloc(s->hw, max_slots, (int)cap, s->npar);
    if (e == cudaSuccess && s->hessian >= 2)
        e = cap > (1 << 28) ? cudaErrorInvalidValue : hw_alloc(s->hwp, max_slots, (int)cap, s->npar);
    for (int i = 0; i < kStepRing && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&s->step_ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_spart, sizeof(double) * 3 * 2 * s->sm_count);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_sticket, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(s->d_sticket, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_sout, sizeof(double) * 3, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->d_sout, s->h_sout, 0);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_fit_stage, sizeof(ToyFit) * max_slots, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_be_stage, sizeof(int64_t) * 2 * max_slots, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_sum_stage, sizeof(double) * max_slots, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_pick, sizeof(int) * max_slots, cudaHostAllocDefault);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_pick, sizeof(int) * max_slots);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_res, sizeof(double) * kResStride * max_slots, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->d_res, s->h_res, 0);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_ev, sizeof(double) * s->n_pad * s->ncols);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_ev, 0, sizeof(double) * s->n_pad * s->ncols, s->stream);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_begin, sizeof(int64_t) * max_slots);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_end, sizeof(int64_t) * max_slots);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_sum_wdm, sizeof(double) * max_slots);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_fits, sizeof(ToyFit) * max_slots);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_counters, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_active, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->d_active, s->h_active, 0);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_done, sizeof(int) * max_slots, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->d_done, s->h_done, 0);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_item_toy, sizeof(int) * s->max_items);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_item_u0, sizeof(int) * s->max_items);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_item_nt, sizeof(int) * s->max_items);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_item_kc, sizeof(KConst) * s->max_items);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_item_dc, sizeof(DConst) * s->max_items);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_unit_item, sizeof(int) * s->max_units);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_unit_tile, sizeof(int) * s->max_units);
    if (e == cudaSuccess) e = gb_malloc(&s->budget, &s->d_unit_sums, sizeof(double) * kAccMax * s->max_units);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_item_toy, 0, sizeof(int) * s->max_items, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_item_u0, 0, sizeof(int) * s->max_items, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_item_nt, 0, sizeof(int) * s->max_items, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_unit_item, 0, sizeof(int) * s->max_units, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_unit_tile, 0, sizeof(int) * s->max_units, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_begin, 0, sizeof(int64_t) * max_slots, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_end, 0, sizeof(int64_t) * max_slots, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_sum_wdm, 0, sizeof(double) * max_slots, s->stream);
    if (e == cudaSuccess) {
        // every slot starts finished (empty); the prepare kernel skips finished slots
        std::vector<ToyFit> idle(max_slots);
        for (auto& F : idle) {
            memset(&F, 0, sizeof F);
            F.phase = kPhDone;
            for (int q = 0; q < kMaxSlots; ++q) F.item[q] = -1;
        }
        e = cudaMemcpyAsync(s->d_fits, idle.data(), sizeof(ToyFit) * max_slots, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    }
    if (e == cudaSuccess) {
        memset(s->h_done, 0, sizeof(int) * max_slots);
        *s->h_active = 0;
        BatchDev d = server_dev(s);
        const int eval_blocks = s->sm_count * 2;
        e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t ec = launch_step(d, kVarPrecompute, false, eval_blocks, s->stream);
            e = cudaStreamEndCapture(s->stream, &s->graph);
            if (e == cudaSuccess) e = ec;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&s->exec, s->graph, 0);
    }
    if (e != cudaSuccess) {
        server_free(s);
        delete s;
        return e == cudaErrorMemoryAllocation ? NLL_ERR_OOM : NLL_ERR_CUDA;
    }
    *out = s;
    return NLL_OK;
}

void nll_server_destroy(nll_server* s)
{
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->cstream) cudaStreamSynchronize(s->cstream);
    server_free(s);
    delete s;
}

const char* nll_server_last_error(const nll_server* s) { return s ? s->err.c_str() : "null server"; }

int nll_server_status(const nll_server* s, int* busy, int* free_slots, int64_t* free_events)
{
    if (!s) return NLL_ERR_ARG;
    int nb = 0;
    for (char c : s->busy) nb += c ? 1 : 0;
    int64_t fe = 0;
    for (auto& r : s->free_ranges) fe += r.second - r.first;
    if (busy) *busy = nb;
    if (free_slots) *free_slots = s->max_slots - nb;
    if (free_events) *free_events = fe;
    return NLL_OK;
}

int nll_server_progress(const nll_server* s, int* steps_in_flight, int* finished)
{
    if (!s) return NLL_ERR_ARG;
    if (steps_in_flight) {
        // the ring holds the events of the last kStepRing steps, newest at step_head - 1; steps
        // complete in order, so count back from the newest until a completed one
        int n = 0;
        for (int k = 1; k <= kStepRing; ++k) {
            cudaEvent_t ev = s->step_ev[(s->step_head - k + kStepRing) % kStepRing];
            cudaError_t q = cudaEventQuery(ev);
            if (q == cudaErrorNotReady) {
                ++n;
                continue;
            }
            if (q != cudaSuccess) return NLL_ERR_CUDA;
            break;
        }
        *steps_in_flight = n;
    }
    if (finished) *finished = finished_count(s);
    return NLL_OK;
}

int nll_server_sync(nll_server* s)
{
    if (!s) return NLL_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cstream);
    return e == cudaSuccess ? NLL_OK : sfail(s, NLL_ERR_CUDA, "server sync: %s", cudaGetErrorString(e));
}

int nll_server_step(nll_server* s, int n_steps)
{
    if (!s || n_steps < 0) return NLL_ERR_ARG;
    if (cudaSetDevice(s->device) != cudaSuccess) return sfail(s, NLL_ERR_CUDA, "cudaSetDevice failed");
    GBNLL_TRACE("server step");
    bool starts = false;
    for (int i = 0; i < s->max_slots; ++i) starts = starts || (s->busy[i] && s->need_start[i]);
    if (starts && n_steps > 0) {
        // start matrices of the requests admitted since the last step: one analytic Hessian
        // pass queued on the step stream ahead of the steps (no wait)
        std::vector<int> pick(s->max_slots, 0);
        for (int i = 0; i < s->max_slots; ++i) pick[i] = s->busy[i] && s->need_start[i];
        cudaError_t e = server_pick(s, s->hw, pick, s->stream, false, s->subsample_start);
        if (e == cudaSuccess)
            e = run_hess_core(server_target(s, s->stream), s->hw, s->cfg, kHmStart, false, nullptr, 0, true, false,
                              s->subsample_start, s->single_start);
        if (e != cudaSuccess) return sfail(s, NLL_ERR_CUDA, "start Hessians: %s", cudaGetErrorString(e));
        for (int i = 0; i < s->max_slots; ++i)
            if (pick[i]) s->need_start[i] = 0;
    }
    for (int i = 0; i < n_steps; ++i) {
        cudaError_t e = cudaGraphLaunch(s->exec, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(s->step_ev[s->step_head], s->stream);
        if (e != cudaSuccess) return sfail(s, NLL_ERR_CUDA, "server step: %s", cudaGetErrorString(e));
        s->step_head = (s->step_head + 1) % kStepRing;
    }
    return NLL_OK;
}

int nll_server_submit(nll_server* s, const double* const* columns, const double* weights, int64_t n_events,
                      const double* theta0, int64_t* request_id)
{
    if (!s || !theta0 || !request_id || n_events < 0) return NLL_ERR_ARG;
    GBNLL_TRACE("server admission");
    if (weights) return sfail(s, NLL_ERR_ARG, "a server serves unweighted fits");
    if (n_events > 0 && !columns) return sfail(s, NLL_ERR_ARG, "null columns");
    for (int d = 0; d < s->ndim && n_events > 0; ++d)
        if (!columns[d]) return sfail(s, NLL_ERR_ARG, "column %d is NULL", d);
    for (int k = 0; k < s->npar; ++k)
        if (!isfinite(theta0[k])) return sfail(s, NLL_ERR_ARG, "start point not finite");
    const int64_t len = std::max<int64_t>((n_events + 1) & ~int64_t(1), 2);
    if (len > s->pool_events) return sfail(s, NLL_ERR_ARG, "more events than the whole pool");
    if (cudaSetDevice(s->device) != cudaSuccess) return sfail(s, NLL_ERR_CUDA, "cudaSetDevice failed");
    int slot = -1;
    for (int i = 0; i < s->max_slots; ++i)
        if (!s->busy[i]) {
            slot = i;
            break;
        }
    int64_t begin = 0;
    if (slot < 0 || !pool_alloc(s, len, &begin)) return sfail(s, NLL_ERR_STATE, "no free slot or pool range");
    // The pool range is free: no queued step or pass reads it, so the request's events go in on
    // the collection stream without waiting for the steps in flight.
    // Host columns the device reads in place (pinned, or pageable with ATS) go into the pool as
    // the statistics kernel reads them, with no host-side staging copy; the rest by cudaMemcpyAsync.
    const cudaStream_t cs = s->cstream;
    cudaError_t e = cudaSuccess;
    const double* src[4] = {nullptr, nullptr, nullptr, nullptr};
    double* dst[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int d = 0; d < s->ndim && e == cudaSuccess && n_events > 0; ++d) {
        double* to = s->d_ev + (size_t)d * s->n_pad + begin;
        if (host_read_in_place(s->device, columns[d])) {
            src[d] = columns[d];
            dst[d] = to;
        } else {
            src[d] = to;
            e = cudaMemcpyAsync(to, columns[d], sizeof(double) * n_events, cudaMemcpyHostToDevice, cs);
        }
    }
    // range check and sum (m - ma) of the request on the device (load-time statistics kernel)
    double sum = 0.0;
    if (e == cudaSuccess && n_events > 0) {
        SArgs sa;
        memset(&sa, 0, sizeof sa);
        for (int d = 0; d < s->ndim; ++d) {
            sa.col[d] = src[d];
            sa.dst[d] = dst[d];
            sa.lo[d] = s->ranges[2 * d];
            sa.hi[d] = s->ranges[2 * d + 1];
        }
        sa.w = nullptr;
        sa.n = n_events;
        sa.ndim = s->ndim;
        sa.partials = s->d_spart;
        sa.ticket = s->d_sticket;
        sa.out = s->d_sout;
        // small blocks (64 threads, 2 warps): they fit beside the step kernels' resident blocks,
        // so an admission does not wait for a step to drain its SM
        const int blocks = (int)std::min<int64_t>(std::max<int64_t>((n_events + 63) / 64, 1), 2 * s->sm_count);
        e = launch_stats(blocks, 64, cs, sa);
    }
    if (e == cudaSuccess && s->kind == kKstar4D && n_events > 0) {
        BArgs ba;
        ba.ctl = s->d_ev + (size_t)kColCtl * s->n_pad + begin;
        ba.ctk = s->d_ev + (size_t)kColCtk * s->n_pad + begin;
        ba.phi = s->d_ev + (size_t)kColPhi * s->n_pad + begin;
        for (int j = 0; j < 13; ++j) ba.out[j] = s->d_ev + (size_t)(kColH0 + j) * s->n_pad + begin;
        ba.n = n_events;
        int blocks = (int)std::min<int64_t>((n_events + 63) / 64, (int64_t)s->sm_count * 16);
        e = launch_basis(std::max(blocks, 1), 64, cs, ba);
    }
    // the copies read the caller's buffers and the check decides the admission: wait for them
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        pool_release(s, begin, len);
        return sfail(s, NLL_ERR_CUDA, "admission: %s", cudaGetErrorString(e));
    }
    if (n_events > 0) {
        if (((volatile double*)s->h_sout)[2] != 0.0) {
            pool_release(s, begin, len);
            return sfail(s, NLL_ERR_ARG, "%.0f event(s) outside the observable ranges", ((volatile double*)s->h_sout)[2]);
        }
        sum = ((volatile double*)s->h_sout)[1];
    }
    // the new fit state, installed on the step stream behind the steps already queued (the
    // staging of this slot was last copied from before the slot's previous fit ran)
    ToyFit& F = s->h_fit_stage[slot];
    init_fit(F, s->cfg, theta0, s->step.data());
    s->h_be_stage[2 * slot] = begin;
    s->h_be_stage[2 * slot + 1] = begin + n_events;
    s->h_sum_stage[slot] = sum;
    e = cudaMemcpyAsync(s->d_fits + slot, &F, sizeof F, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_begin + slot, s->h_be_stage + 2 * slot, sizeof(int64_t), cudaMemcpyHostToDevice,
                            s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_end + slot, s->h_be_stage + 2 * slot + 1, sizeof(int64_t), cudaMemcpyHostToDevice,
                            s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_sum_wdm + slot, s->h_sum_stage + slot, sizeof(double), cudaMemcpyHostToDevice,
                            s->stream);
    if (e != cudaSuccess) {
        pool_release(s, begin, len);
        return sfail(s, NLL_ERR_CUDA, "admission: %s", cudaGetErrorString(e));
    }
    s->slot_begin[slot] = begin;
    s->slot_len[slot] = len;
    s->slot_nev[slot] = n_events;
    // strategy 2: the start matrix comes from one analytic Hessian pass over every request
    // admitted since the last step, queued by the next nll_server_step before its first step
    s->need_start[slot] = s->cfg.strategy == 2 ? 1 : 0;
    s->h_done[slot] = 0;
    __atomic_add_fetch(s->h_active, 1, __ATOMIC_SEQ_CST);
    s->busy[slot] = 1;
    s->slot_id[slot] = s->next_id;
    *request_id = s->next_id++;
    return NLL_OK;
}

int nll_server_poll(nll_server* s, int64_t* ids_out, fit_result* results, int max_results, int* n_out)
{
    if (!s || !n_out || max_results < 0 || (max_results > 0 && (!ids_out || !results))) return NLL_ERR_ARG;
    *n_out = 0;
    GBNLL_TRACE("server collection");
    if (cudaSetDevice(s->device) != cudaSuccess) return sfail(s, NLL_ERR_CUDA, "cudaSetDevice failed");
    // fits whose done flag is set: their final state is in device memory and no step changes it
    std::vector<int> pick(s->max_slots, 0);
    int np = 0;
    for (int i = 0; i < s->max_slots && np < max_results; ++i)
        if (s->busy[i] && ((volatile int*)s->h_done)[i]) {
            pick[i] = 1;
            s->h_pick[np++] = i;
        }
    if (np == 0) {
        // nothing finished: report a failed step, if any, without waiting for the others
        cudaError_t q = cudaStreamQuery(s->stream);
        if (q != cudaSuccess && q != cudaErrorNotReady)
            return sfail(s, NLL_ERR_CUDA, "server step: %s", cudaGetErrorString(q));
        return NLL_OK;
    }
    const cudaStream_t cs = s->cstream;
    cudaError_t e = cudaSuccess;
    if (s->hessian >= 2) {  // Newton polish and covariance with the analytic Hessian
        e = server_pick(s, s->hwp, pick, cs, true);
        if (e == cudaSuccess) e = polish_core(server_target(s, cs), s->hwp, s->cfg, s->hessian, true);
        if (e != cudaSuccess) return sfail(s, NLL_ERR_CUDA, "Newton polish: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(s->d_pick, s->h_pick, sizeof(int) * np, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = launch_pack_results(s->d_fits, s->d_pick, np, s->npar, s->cfg.nf, s->d_res, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return sfail(s, NLL_ERR_CUDA, "result collection: %s", cudaGetErrorString(e));
    for (int k = 0; k < np; ++k) {
        const int i = s->h_pick[k];
        fill_result_packed(s->h_res + (size_t)k * kResStride, s->cfg, results[k]);
        ids_out[k] = s->slot_id[i];
        s->busy[i] = 0;
        s->h_done[i] = 0;
        pool_release(s, s->slot_begin[i], s->slot_len[i]);
    }
    *n_out = np;
    return NLL_OK;
}

int nll_server_cancel(nll_server* s, int64_t request_id)
{
    if (!s) return NLL_ERR_ARG;
    int slot = -1;
    for (int i = 0; i < s->max_slots; ++i)
        if (s->busy[i] && s->slot_id[i] == request_id) slot = i;
    if (slot < 0) return sfail(s, NLL_ERR_ARG, "no fit with request id %lld in the server", (long long)request_id);
    if (cudaSetDevice(s->device) != cudaSuccess) return sfail(s, NLL_ERR_CUDA, "cudaSetDevice failed");
    // the queued steps may still read the fit's events: let them finish, then mark the fit
    // finished on the device so no later step or pass touches it, and free its slot and range
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cstream);
    if (e == cudaSuccess) {
        const int done_phase = kPhDone;
        e = cudaMemcpyAsync(&s->d_fits[slot].phase, &done_phase, sizeof done_phase, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    }
    if (e != cudaSuccess) return sfail(s, NLL_ERR_CUDA, "cancel: %s", cudaGetErrorString(e));
    if (!((volatile int*)s->h_done)[slot]) __atomic_sub_fetch(s->h_active, 1, __ATOMIC_SEQ_CST);
    s->busy[slot] = 0;
    s->h_done[slot] = 0;
    s->need_start[slot] = 0;
    pool_release(s, s->slot_begin[slot], s->slot_len[slot]);
    return NLL_OK;
}

}  // extern "C"
