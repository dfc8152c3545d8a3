// batch_internal.h -- types and host helpers shared by the batched-fit code (batch.cu) and
// the server (server.cu): the device fit state of one toy, the minimiser settings, the
// device work arrays of a step, and the analytic-Hessian work arrays and passes.  Not part
// of the public C ABI (include/gbnll.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/gbnll.h"
#include "gbnll_internal.h"
#include "hess_device.cuh"

namespace gbnll {

constexpr int kNP = 18;                 // largest parameter count
constexpr int kMaxSlots = 2 * kNP + 1;  // trial point + stencil points per toy and step
constexpr int kEvalThreads = 128;
constexpr int kUpdWarps = 4;

enum Phase : int { kPhInit = 0, kPhSearch = 1, kPhHess = 2, kPhDone = 3 };

// Derivative constants of one parameter point (device copy of the host Hoist fields).
struct DConst {
    double mu, sigma, alpha, f, ma, b0, b2, dlnN1_dmu, dlnN1_dsig, dlnN2t_dal, dlnNc[3];
    double lnb1, d2lnN1[3], d2lnN2t_dal2;  // for the analytic Hessian
    int ok;
};

// Minimiser state of one toy (device).
struct ToyFit {
    int phase, iter, n_eval, status, first;
    int vset;  // the start matrix V came from the analytic Hessian (strategy 2)
    int nitem;  // item slots [0, nitem) written by the last prepare (the rest are unused)
    // Newton polish with the analytic Hessian after the loop (hessian 2 / 3)
    int pol;                  // > 0 while polishing
    double lam, f_acc;        // step fraction; NLL at the accepted point
    double th_acc[kNP];       // accepted point (all parameters)
    double dN[kNP];           // Newton direction H^-1 g (free components, external)
    double f, ft, edm, alpha, gp;
    double x[kNP], g[kNP], p[kNP], xt[kNP], sint[kNP], hstep[kNP];
    double th[kNP];    // external parameters of the accepted point (all npar)
    double gext[kNP];  // external gradient (free components) at the accepted point
    double V[kNP * kNP];
    double gsten[2 * kNP][kNP];
    double cov[kNP * kNP];
    double err[kNP];
    int item[kMaxSlots];
};

struct FitConfig {
    int kind, npar, nf, strategy, hessian, max_iter;
    double tol_edm;
    double ranges[8];
    int idx[kNP];
    int bounded[kNP];
    double lo[kNP], hi[kNP];
};

struct BatchDev {
    int n_toys, tile_pairs;        // tile_pairs = 0: one unit per item
    const int* step_tp;            // or NULL: the tile of this step (a device step of the fit loop
                                   // shrinks it once few toys are left), in place of tile_pairs
    const int64_t* ev_begin;       // per toy, even
    const int64_t* ev_end;         // per toy, exclusive
    const double* sum_wdm;         // per toy: sum w (m - ma)
    KArgs cols;                    // column pointers and weights
    ToyFit* fits;
    int* counters;                 // [0] items, [1] units, [2] next unit
    int* n_active;                 // toys not yet done (mapped host memory)
    int* done_flags;               // per toy, set to 1 when it finishes (mapped), or NULL
    int* item_toy;
    int* item_u0;
    int* item_nt;
    KConst* item_kc;
    DConst* item_dc;
    int* unit_item;
    int* unit_tile;
    double* unit_sums;             // [max_units][kAccMax]
    int max_items, max_units;
    FitConfig cfg;
};


// analytic Hessian pass over the toys (paper Sec. 2.1)
constexpr int kHessUnitEvents = 512;  // 4 shared-memory tiles: the units of 1000 toys of 2000 events
                                       // spread over the SMs within 4 % (1024: 7 %)

enum HessMode : int { kHmEval = 0, kHmStart = 1, kHmCov = 2, kHmSandwich = 3 };

// per toy, the assembled Hessian pass (stored entry-major, [entry][toy]): nll, grad[NP],
// H[NP x NP], W[NP x NP], the non-positive-density count
constexpr int kAsmEntries = 2 + kNP + 2 * kNP * kNP;

// doubles per toy of a packed result: th[npar] | err[nf] | cov[nf x nf] | nll, edm, n_eval, n_iter, status
constexpr int kResStride = 2 * kNP + kNP * kNP + 5;

// Work arrays of the analytic Hessian pass: units of kHessUnitEvents events of the selected
// toys, per-toy constants and results, per-unit slot sums, the slot table, a selection mask
// and the polish counter.
struct HessWork {
    bool ready = false;
    int cap_toys = 0, cap_units = 0, np = 0, n_units = 0;
    int layout_key = -1;  // slot table on the device: kind, weights, W
    int* d_unit_toy = nullptr;
    int64_t* d_unit_e0 = nullptr;
    int* d_toy_u0 = nullptr;
    int* d_toy_nu = nullptr;
    HConst* d_hc = nullptr;
    HessTerms* d_ht = nullptr;
    int* d_hok = nullptr;
    double* d_unit_sums = nullptr;
    double* d_tot = nullptr;   // slot totals per toy
    double* d_asm = nullptr;   // assembled NLL, gradient, H, W per toy
    uint16_t* d_slot_of = nullptr;
    double* d_thetas = nullptr;
    double* d_out = nullptr;
    int* d_status = nullptr;
    int* d_sel = nullptr;
    int* h_npol = nullptr;  // mapped: toys that proposed a polish step in the last pass
    int* d_npol = nullptr;
    // pinned staging of the unit lists and the event behind their last copies
    int* h_unit_toy = nullptr;
    int64_t* h_unit_e0 = nullptr;
    int* h_toy_u0 = nullptr;
    int* h_toy_nu = nullptr;
    int* h_sel = nullptr;
    cudaEvent_t staged_ev = nullptr;
    bool staged_pending = false;
    DevBudget* budget = nullptr;  // the owner's device-memory count (kept by hw_free)
};

// The sample and fit states a Hessian pass works on.
struct HessTarget {
    int kind, variant, sm_count, n_toys;
    int max_bps;  // event-pass blocks per SM at most (0: as many as fit, up to 4)
    bool weighted;
    HEv ev;
    const int64_t* d_begin;
    const int64_t* d_end;
    const double* d_sum_wdm;
    ToyFit* d_fits;
    cudaStream_t stream;
};

// ---- host helpers (batch.cu) ----
void hw_free(HessWork& w);
cudaError_t hw_alloc(HessWork& w, int cap_toys, int cap_units, int np);
// Unit lists for toys t with events [begin[t], end[t]); toys with sel[t] == 0 get no units
// (sel empty: every toy).  With wait, returns once they are on the device; without, once the
// copies (from pinned staging) are queued on the stream.
// With subsample, a toy takes the first of its 1024-event units when it has up to 8, else 4
// units spread evenly over its events (a start matrix; see run_hess_core).
cudaError_t hw_set_units(HessWork& w, const std::vector<int64_t>& begin, const std::vector<int64_t>& end,
                         const std::vector<int>& sel, cudaStream_t stream, bool wait = true,
                         bool subsample = false);
// One Hessian pass (mode HessMode); use_sel restricts it to the toys hw_set_units selected.
// With wait, returns once the pass has finished; without, once it is queued on T.stream.
// subsample: the unit lists cover part of each toy's events (hw_set_units with subsample); the
// slot sums are scaled by events / events covered before the assembly (start matrices only).
// single: the event pass in single precision (start matrices only).
cudaError_t run_hess_core(const HessTarget& T, HessWork& w, const FitConfig& cfg, int mode, bool want_w2,
                          const double* thetas, int pass, bool use_sel, bool wait = true, bool subsample = false,
                          bool single = false);
// Newton polish passes with the analytic Hessian at the final points of the finished toys.
// speculate: queue passes 0 and 1 without waiting in between (large batches).
cudaError_t polish_core(const HessTarget& T, HessWork& w, const FitConfig& cfg, int hessian, bool use_sel,
                        bool speculate = false);
void setup_config(FitConfig& c, int np, const double* lo, const double* hi, const double* step, const int* fixed,
                  const fit_options& opt);
void init_fit(ToyFit& F, const FitConfig& c, const double* th0, const double* step);
void fill_result(const ToyFit& F, const FitConfig& c, fit_result& r);
void fill_result_packed(const double* p, const FitConfig& c, fit_result& r);
// The device tables of the batched kernels on `device` (current), uploaded once.
cudaError_t ensure_btab(int device);
cudaError_t launch_eval(int kind, int var, bool w, int blocks, cudaStream_t s, const BatchDev& b);
// One device step (counter reset, prepare, evaluate, update) on stream s, for graph capture.
cudaError_t launch_step(const BatchDev& d, int var, bool weighted, int eval_blocks, cudaStream_t s);
cudaError_t launch_step_eval(const BatchDev& d, int var, bool weighted, int eval_blocks, cudaStream_t s);
cudaError_t launch_step_update(const BatchDev& d, cudaStream_t s);
// Results of n toys packed for the host, kResStride doubles each: toys idx[0..n) (device
// array), or 0 .. n-1 when idx is NULL.
cudaError_t launch_pack_results(const ToyFit* fits, const int* idx, int n, int np, int nf, double* res,
                                cudaStream_t s);

}  // namespace gbnll
