// hc_tune.cu -- the autotuner: search parameters per (alphabet size,
// pattern length) cell, measured on the batched kernels.
//
// The paper chooses q and alpha per text and pattern length from its own
// measurements (Sec. 4, Tables 1-3) and leaves the word width hard-coded.
// Here the same choice is measured on this GPU, together with the launch
// options of the scan (window starts per lane, staged or direct mode): for
// each cell a calibration text (i.i.d. uniform over sigma symbols, drawn on
// the device from a counter-based generator) and a pattern copied from it
// are searched as a one-query batch for every candidate, and the fastest
// candidate is kept.  An empty table falls back to the paper's tables.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "hc_batch_internal.h"

namespace hc {

constexpr uint32_t kTunerMagic = 0x48435455u;  // "HCTU"
constexpr uint64_t kScreenBytes = 8ull << 20;  // text per screening run
constexpr size_t kFinalists = 8;                // candidates timed on the whole text
constexpr int kTunePatterns = 5;                 // patterns the finalists are timed on

struct Tuner {
  uint32_t magic = kTunerMagic;
  std::mutex mu;
  std::vector<hc_tune_entry> cells;  // sorted by (sigma, m)
};

Tuner* as_tuner(const hc_tuner* t) {
  auto* p = reinterpret_cast<Tuner*>(const_cast<hc_tuner*>(t));
  return (p != nullptr && p->magic == kTunerMagic) ? p : nullptr;
}

namespace {

// The paper's best-measured (q, alpha) of HC (Tables 1-3) for its genome,
// protein and English texts at m = 8, 16, ..., 1024.
constexpr int kPaperRows = 8;
constexpr int kPaperQ[3][kPaperRows] = {{4, 6, 6, 6, 6, 6, 6, 8},
                                        {3, 3, 3, 6, 3, 3, 4, 4},
                                        {3, 3, 6, 6, 3, 3, 4, 4}};
constexpr int kPaperAlpha[3][kPaperRows] = {{12, 12, 12, 12, 12, 12, 12, 12},
                                            {11, 11, 11, 12, 11, 11, 12, 12},
                                            {11, 11, 12, 12, 11, 11, 12, 12}};

QueryParams paper_params(double sigma, uint64_t m) {
  const int col = sigma <= 8.0 ? 0 : (sigma <= 40.0 ? 1 : 2);
  const double lm = std::log2(static_cast<double>(std::max<uint64_t>(m, 1)));
  int row = 0;
  double best = 1e30;
  for (int r = 0; r < kPaperRows; ++r) {  // nearest m on a log scale, the smaller on a tie
    const double d = std::fabs(lm - (3 + r));
    if (d < best) {
      best = d;
      row = r;
    }
  }
  QueryParams p;
  p.q = static_cast<int>(std::min<uint64_t>(kPaperQ[col][row], std::max<uint64_t>(m, 1)));
  p.alpha = kPaperAlpha[col][row];
  return p;
}

// Shared memory of the batched scan for one staged query (the layout of
// plan_finish), against the opt-in limit of sm_100-class devices.
bool staged_fits(int L, uint64_t m, int alpha) {
  const uint64_t C = 32ull * static_cast<uint64_t>(std::max(L, 1));
  const uint64_t stage = stage_bytes_for(static_cast<uint32_t>(C), m, false);
  const uint64_t x = m <= 4096 ? ((m + 15) & ~uint64_t(15)) : 0;
  const uint64_t smem = (4ull << alpha) + x + uint64_t(kSlots) * kThreads * 4 + uint64_t(kWarps) * 2 * stage;
  return m <= static_cast<uint64_t>(kMaxStagedM) && smem + 2048 <= 232448;
}

// n bytes i.i.d. uniform over sigma symbols 'A', 'A'+1, ...: byte i is
// drawn from splitmix64(seed + i) (Steele, Lea and Flood, 2014) by
// multiply-shift range reduction.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void hc_tune_text_kernel(uint8_t* y, unsigned long long n, int sigma, unsigned long long seed) {
  const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
  for (unsigned long long i = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x; i < n;
       i += stride) {
    const uint64_t r = splitmix64(seed + i) >> 32;
    y[i] = static_cast<uint8_t>(65u + static_cast<uint32_t>((r * static_cast<uint64_t>(sigma)) >> 32));
  }
}

void sort_cells(std::vector<hc_tune_entry>& c) {
  std::sort(c.begin(), c.end(), [](const hc_tune_entry& a, const hc_tune_entry& b) {
    return a.sigma != b.sigma ? a.sigma < b.sigma : a.m < b.m;
  });
}

void put_cell(Tuner* t, const hc_tune_entry& e) {
  for (auto& c : t->cells)
    if (c.sigma == e.sigma && c.m == e.m) {
      c = e;
      return;
    }
  t->cells.push_back(e);
  sort_cells(t->cells);
}

// Device buffers reused across the candidates of a calibration.
struct Scratch {
  SearchArgs* args = nullptr;
  BatchTile* tiles = nullptr;
  size_t tiles_cap = 0;
  EmitTile* etiles = nullptr;
  size_t etiles_cap = 0;
  unsigned long long* counter = nullptr;  // [0, kMaxScanClasses) work counters, then the count
  uint32_t* filters = nullptr;
  size_t filters_cap = 0;
  uint8_t* ws = nullptr;
  size_t ws_cap = 0;
  uint8_t* fx = nullptr;        // single path: filter words + pattern (device)
  size_t fx_cap = 0;
  uint8_t* host = nullptr;      // pinned staging of launch tables / filters
  size_t host_cap = 0;
  ~Scratch() {
    cudaFree(args);
    cudaFree(tiles);
    cudaFree(etiles);
    cudaFree(counter);
    cudaFree(filters);
    cudaFree(ws);
    cudaFree(fx);
    cudaFreeHost(host);
  }
};

int grow_host(Scratch& sc, size_t need) {
  if (need <= sc.host_cap && sc.host != nullptr) return HC_OK;
  cudaFreeHost(sc.host);
  sc.host = nullptr;
  sc.host_cap = 0;
  const size_t n = std::max<size_t>(need * 2, 1 << 16);
  void* v = nullptr;
  cudaError_t e = cudaHostAlloc(&v, n, cudaHostAllocDefault);
  if (e != cudaSuccess) return cuda_error(e, "cudaHostAlloc(tuner staging)");
  sc.host = static_cast<uint8_t*>(v);
  sc.host_cap = n;
  return HC_OK;
}

template <typename T>
int grow(T** p, size_t* cap, size_t need, const char* what) {
  if (need <= *cap && *p != nullptr) return HC_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  void* v = nullptr;
  const size_t n = std::max<size_t>(need, 1) * 2;
  cudaError_t e = cudaMalloc(&v, n * sizeof(T));
  if (e != cudaSuccess) return cuda_error(e, what);
  *p = static_cast<T*>(v);
  *cap = n;
  return HC_OK;
}

// Best of `reps` timed runs (after one untimed) of the one-query batch of
// (x, y) with parameters p; +inf when the parameters do not fit.
int time_candidate(Scratch& sc, int dev, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n,
                   const QueryParams& p, int reps, bool warm, cudaStream_t stream, cudaEvent_t e0,
                   cudaEvent_t e1, double* seconds, int* lane_bytes, int* mode) {
  *seconds = INFINITY;
  hc_batch_query Q{};
  Q.x_dev = x;
  Q.m = m;
  Q.y_dev = y;
  Q.n = n;
  Q.q = p.q;
  Q.alpha = p.alpha;
  Q.count_dev = reinterpret_cast<uint64_t*>(sc.counter + kMaxScanClasses);
  Q.lane_bytes = p.lane_bytes;
  Q.mode = p.mode;
  BatchPlan plan;
  if (plan_add_query(plan, Q, 0, p, record_bytes_for(n, dev), "hc_tuner_calibrate") != HC_OK ||
      plan_finish(plan, dev, "hc_tuner_calibrate") != HC_OK) {
    clear_error();  // does not fit: skipped
    return HC_OK;
  }
  int rc = grow(&sc.tiles, &sc.tiles_cap, plan.tiles.size(), "cudaMalloc(tuner tiles)");
  if (rc == HC_OK) rc = grow(&sc.etiles, &sc.etiles_cap, plan.etiles.size(), "cudaMalloc(tuner emit tiles)");
  if (rc == HC_OK) rc = grow(&sc.filters, &sc.filters_cap, plan.filter_words, "cudaMalloc(tuner filters)");
  if (rc == HC_OK) rc = grow(&sc.ws, &sc.ws_cap, plan.ws_bytes, "cudaMalloc(tuner workspace)");
  if (rc != HC_OK) return rc;
  plan_bind(plan, sc.filters, sc.ws);
  // the tables go through pinned staging (pageable copies would synchronise);
  // the previous candidate's copies have completed (its runs were waited for)
  const size_t tb = plan.tiles.size() * sizeof(BatchTile), eb = plan.etiles.size() * sizeof(EmitTile);
  rc = grow_host(sc, sizeof(SearchArgs) + tb + eb);
  if (rc != HC_OK) return rc;
  std::memcpy(sc.host, plan.args.data(), sizeof(SearchArgs));
  std::memcpy(sc.host + sizeof(SearchArgs), plan.tiles.data(), tb);
  std::memcpy(sc.host + sizeof(SearchArgs) + tb, plan.etiles.data(), eb);
  cudaError_t e = cudaMemcpyAsync(sc.args, sc.host, sizeof(SearchArgs), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && tb)
    e = cudaMemcpyAsync(sc.tiles, sc.host + sizeof(SearchArgs), tb, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && eb)
    e = cudaMemcpyAsync(sc.etiles, sc.host + sizeof(SearchArgs) + tb, eb, cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(tuner tables)");
  rc = batch_grids(plan, dev);
  if (rc != HC_OK) return rc;
  const BatchLaunch L = make_launch(plan, sc.args, sc.tiles, sc.etiles, sc.counter);
  if (warm) rc = launch_batch(L, stream);
  double best = INFINITY;
  for (int r = 0; r < reps && rc == HC_OK; ++r) {
    cudaEventRecord(e0, stream);
    rc = launch_batch(L, stream);
    cudaEventRecord(e1, stream);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventSynchronize(tuner)");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms * 1e-3);
  }
  if (rc != HC_OK) return rc;
  *seconds = best;
  *lane_bytes = plan.args[0].records ? plan.args[0].L : p.lane_bytes;
  *mode = plan.args[0].stages > 0 ? HC_MODE_STAGED : HC_MODE_DIRECT;
  return HC_OK;
}

// The same for the single-search path: a host-built filter (hc_preprocess)
// and the two kernels of hc_search_ex (dense, staged or direct scan, emit).
int time_candidate_single(Scratch& sc, int dev, const std::vector<uint8_t>& xh, const uint8_t* y, uint64_t n,
                          const QueryParams& p, int reps, bool warm, cudaStream_t stream, cudaEvent_t e0,
                          cudaEvent_t e1, double* seconds, int* lane_bytes, int* mode) {
  *seconds = INFINITY;
  hc_filter* fh = nullptr;
  if (hc_preprocess(xh.data(), xh.size(), p.q, p.alpha, &fh) != HC_OK) {
    clear_error();
    return HC_OK;
  }
  Filter* f = as_filter(fh);
  hc_search_opts o{};
  o.struct_size = sizeof o;
  o.lane_bytes = p.lane_bytes;
  o.mode = p.mode;
  o.sentinel = p.sentinel;
  o.bitmap = p.bitmap;
  SearchPlan sp;
  if (plan_search(f, n, 0, &o, dev, &sp) != HC_OK) {
    clear_error();
    hc_filter_free(fh);
    return HC_OK;
  }
  // the filter words and the pattern through pinned staging into a reused
  // device buffer (no per-candidate allocation)
  const size_t fbytes = (f->F.size() * 4 + 15) & ~size_t(15);
  int rc = grow(&sc.ws, &sc.ws_cap, sp.ws_bytes, "cudaMalloc(tuner workspace)");
  if (rc == HC_OK) rc = grow(&sc.fx, &sc.fx_cap, fbytes + f->x.size(), "cudaMalloc(tuner filter)");
  if (rc == HC_OK) rc = grow_host(sc, fbytes + f->x.size());
  if (rc == HC_OK) {
    std::memcpy(sc.host, f->F.data(), f->F.size() * 4);
    std::memcpy(sc.host + fbytes, f->x.data(), f->x.size());
    cudaError_t e = cudaMemcpyAsync(sc.fx, sc.host, fbytes + f->x.size(), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) rc = cuda_error(e, "cudaMemcpyAsync(tuner filter)");
  }
  const uint32_t* F_dev = reinterpret_cast<const uint32_t*>(sc.fx);
  const uint8_t* x_dev = sc.fx + fbytes;
  uint64_t* count = reinterpret_cast<uint64_t*>(sc.counter + kMaxScanClasses);
  if (rc == HC_OK && warm) rc = launch_planned_filter_ptrs(f, sp, F_dev, x_dev, y, n, nullptr, 0, count, sc.ws, stream);
  double best = INFINITY;
  for (int r = 0; r < reps && rc == HC_OK; ++r) {
    cudaEventRecord(e0, stream);
    rc = launch_planned_filter_ptrs(f, sp, F_dev, x_dev, y, n, nullptr, 0, count, sc.ws, stream);
    cudaEventRecord(e1, stream);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      rc = cuda_error(e, "cudaEventSynchronize(tuner)");
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms * 1e-3);
  }
  hc_filter_free(fh);
  if (rc != HC_OK) return rc;
  *seconds = best;
  *lane_bytes = sp.L;
  *mode = sp.kind;
  return HC_OK;
}

int calibrate_cell(Tuner* t, Scratch& sc, int dev, const uint8_t* y, uint64_t n, int sigma, uint64_t m,
                   uint64_t seed, int path, cudaStream_t stream, cudaEvent_t e0, cudaEvent_t e1) {
  // the patterns: m bytes of the text at seeded offsets (the screening uses
  // the first; the finalists are timed on all of them, so that one pattern's
  // particular q-grams do not decide the cell)
  const uint8_t* xs[kTunePatterns];
  std::vector<uint8_t> xh[kTunePatterns];
  for (int k = 0; k < kTunePatterns; ++k) {
    const uint64_t off = ((seed + 7919ull * k) * 0x9E3779B97F4A7C15ull ^ m * 0xBF58476D1CE4E5B9ull) % (n - m + 1);
    xs[k] = y + off;
    xh[k].resize(m);
    if (path == HC_TUNE_SINGLE) {
      cudaError_t e = cudaMemcpy(xh[k].data(), xs[k], m, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(calibration pattern)");
    }
  }
  // timed on the first nn bytes of the text with `npat` patterns: reps runs
  // each (after an untimed one when warm), the patterns' best times summed
  auto time_it = [&](const QueryParams& p, uint64_t nn, int reps, bool warm, double* s, int* L, int* mode,
                     int npat = kTunePatterns) -> int {
    double total = 0;
    for (int k = 0; k < npat; ++k) {
      double sk = INFINITY;
      const int rc = path == HC_TUNE_SINGLE
                         ? time_candidate_single(sc, dev, xh[k], y, nn, p, reps, warm, stream, e0, e1, &sk, L, mode)
                         : time_candidate(sc, dev, xs[k], m, y, nn, p, reps, warm, stream, e0, e1, &sk, L, mode);
      if (rc != HC_OK) return rc;
      total += sk;
      if (!std::isfinite(sk)) break;
    }
    *s = total;
    return HC_OK;
  };
  // screening: every (q, alpha) once on a prefix of the text (a poor
  // candidate can be orders of magnitude slower than a good one: every
  // window passing the first test and walking far); the best few are then
  // timed on the whole text
  struct Cand {
    double s;
    QueryParams p;
  };
  std::vector<Cand> screened;
  const uint64_t n_screen = std::min<uint64_t>(n, std::max<uint64_t>(kScreenBytes, 64 * m));
  for (int q = 1; q <= static_cast<int>(std::min<uint64_t>(8, m)); ++q)
    for (int alpha = 8; alpha <= 13; ++alpha) {
      QueryParams p;
      p.q = q;
      p.alpha = alpha;
      double s = INFINITY;
      int L = 0, mode = 0;
      int rc = time_it(p, n_screen, 1, false, &s, &L, &mode, 1);
      if (rc != HC_OK) return rc;
      if (std::isfinite(s)) screened.push_back({s, p});
    }
  if (screened.empty()) return set_error(HC_ERR_ARG, "hc_tuner_calibrate: no candidate fits");
  std::sort(screened.begin(), screened.end(), [](const Cand& a, const Cand& b) { return a.s < b.s; });
  double best = INFINITY;
  QueryParams bp;
  int best_L = 0, best_mode = 0;
  for (size_t k = 0; k < screened.size() && k < kFinalists; ++k) {
    double s = INFINITY;
    int L = 0, mode = 0;
    int rc = time_it(screened[k].p, n, 3, true, &s, &L, &mode);
    if (rc != HC_OK) return rc;
    if (s < best) {
      best = s;
      bp = screened[k].p;
      best_L = L;
      best_mode = mode;
    }
  }
  if (!std::isfinite(best)) return set_error(HC_ERR_ARG, "hc_tuner_calibrate: no candidate fits");
  const int L0 = best_L;
  for (int mode : {HC_MODE_STAGED, HC_MODE_DIRECT, HC_MODE_DENSE})
    for (int L : {L0 / 2, L0, L0 * 3 / 2, L0 * 2}) {
      if (L < 1 || L > 4096 || (mode == best_mode && L == L0)) continue;
      if (L == L0 * 3 / 2 && mode != HC_MODE_DENSE) continue;  // wider dense lanes: fewer CTAs, larger steps
      if (mode == HC_MODE_DENSE && (path != HC_TUNE_SINGLE || static_cast<uint64_t>(bp.q) != m)) continue;
      QueryParams p = bp;
      p.lane_bytes = L;
      p.mode = mode;
      double s = INFINITY;
      int Lr = 0, mr = 0;
      int rc = time_it(p, n, 3, true, &s, &Lr, &mr);
      if (rc != HC_OK) return rc;
      if (s < best) {
        best = s;
        best_L = Lr;
        best_mode = mr;
      }
    }
  // the sentinel form of the staged scan (single searches): kept where it
  // is faster
  int best_sentinel = 0;
  if (path == HC_TUNE_SINGLE && best_mode == HC_MODE_STAGED) {
    QueryParams p = bp;
    p.lane_bytes = best_L;
    p.mode = HC_MODE_STAGED;
    p.sentinel = 1;
    double s = INFINITY;
    int Lr = 0, mr = 0;
    int rc = time_it(p, n, 3, true, &s, &Lr, &mr);
    if (rc != HC_OK) return rc;
    if (s < best && mr == HC_MODE_STAGED) {
      best = s;
      best_sentinel = 1;
    }
  }
  // the bitmap form of the dense scan (single searches, m = q): kept where
  // it is faster (patterns with many occurrences), at the lane width found
  // above or twice or half of it
  int best_bitmap = 0;
  if (path == HC_TUNE_SINGLE && best_mode == HC_MODE_DENSE) {
    const int Lb = best_L;
    for (int L : {Lb, Lb * 2, Lb / 2}) {
      if (L < 2 || L > 256) continue;
      QueryParams p = bp;
      p.lane_bytes = L;
      p.mode = HC_MODE_DENSE;
      p.bitmap = 1;
      double s = INFINITY;
      int Lr = 0, mr = 0;
      int rc = time_it(p, n, 3, true, &s, &Lr, &mr);
      if (rc != HC_OK) return rc;
      if (s < best && mr == HC_MODE_DENSE) {
        best = s;
        best_bitmap = 1;
        best_L = Lr;
      }
    }
  }
  hc_tune_entry c{};
  c.sigma = sigma;
  c.m = m;
  c.q = bp.q;
  c.alpha = bp.alpha;
  c.lane_bytes = best_L;
  c.mode = best_mode;
  c.sentinel = best_sentinel;
  c.bitmap = best_bitmap;
  c.gbps = static_cast<double>(n) * kTunePatterns / best / 1e9;
  std::lock_guard<std::mutex> lock(t->mu);
  put_cell(t, c);
  return HC_OK;
}

}  // namespace

QueryParams tuner_lookup(const Tuner* t, double sigma, uint64_t m) {
  m = std::max<uint64_t>(m, 1);
  if (sigma <= 0) sigma = 4;
  hc_tune_entry best{};
  bool found = false;
  if (t != nullptr) {
    std::lock_guard<std::mutex> lock(const_cast<Tuner*>(t)->mu);
    // nearest alphabet size, then nearest pattern length, on log scales
    double ds = 1e30;
    int col = 0;
    for (const auto& c : t->cells) {
      const double d = std::fabs(std::log(static_cast<double>(c.sigma)) - std::log(sigma));
      if (d < ds - 1e-12) {
        ds = d;
        col = c.sigma;
      }
    }
    double dm = 1e30;
    for (const auto& c : t->cells) {
      if (c.sigma != col) continue;
      const double d = std::fabs(std::log(static_cast<double>(c.m)) - std::log(static_cast<double>(m)));
      if (d < dm - 1e-12) {
        dm = d;
        best = c;
        found = true;
      }
    }
  }
  if (!found) return paper_params(sigma, m);
  QueryParams p;
  p.q = static_cast<int>(std::min<uint64_t>(best.q, m));
  p.alpha = best.alpha;
  p.lane_bytes = best.lane_bytes;
  p.mode = best.mode;
  p.sentinel = best.sentinel;
  p.bitmap = best.bitmap;
  if (best.m != m) {
    // launch options measured for another length: keep them only where they
    // still fit (the staged form's buffers grow with m; the dense form needs
    // m = q)
    if ((p.mode == HC_MODE_STAGED && !staged_fits(p.lane_bytes, m, p.alpha)) ||
        (p.mode == HC_MODE_DENSE && static_cast<uint64_t>(p.q) != m)) {
      p.mode = HC_MODE_AUTO;
      p.lane_bytes = 0;
      p.sentinel = 0;
      p.bitmap = 0;
    }
  }
  return p;
}

}  // namespace hc

using namespace hc;

extern "C" {

int hc_tuner_create(hc_tuner** out) {
  clear_error();
  if (out == nullptr) return set_error(HC_ERR_ARG, "hc_tuner_create: out is NULL");
  Tuner* t = new (std::nothrow) Tuner();
  if (t == nullptr) return set_error(HC_ERR_NOMEM, "hc_tuner_create: out of host memory");
  *out = reinterpret_cast<hc_tuner*>(t);
  return HC_OK;
}

void hc_tuner_free(hc_tuner* tp) {
  Tuner* t = as_tuner(tp);
  if (t == nullptr) return;
  t->magic = 0;
  delete t;
}

int hc_tuner_calibrate(hc_tuner* tp, const int* sigmas, size_t nsigma, const uint64_t* ms, size_t nm,
                       uint64_t text_bytes, uint64_t seed, int path, hc_stream_t stream_) {
  clear_error();
  Tuner* t = as_tuner(tp);
  if (t == nullptr) return set_error(HC_ERR_ARG, "hc_tuner_calibrate: invalid tuner");
  if ((sigmas == nullptr && nsigma > 0) || (ms == nullptr && nm > 0))
    return set_error(HC_ERR_ARG, "hc_tuner_calibrate: NULL list");
  for (size_t i = 0; i < nsigma; ++i)
    if (sigmas[i] < 1 || sigmas[i] > 190) return set_error(HC_ERR_ARG, "hc_tuner_calibrate: sigma out of [1, 190]");
  for (size_t i = 0; i < nm; ++i)
    if (ms[i] < 1 || ms[i] > 65536 || ms[i] > text_bytes)
      return set_error(HC_ERR_ARG, "hc_tuner_calibrate: m out of [1, min(65536, text_bytes)]");
  if (text_bytes < 1 || text_bytes > (uint64_t(1) << 34))
    return set_error(HC_ERR_ARG, "hc_tuner_calibrate: text_bytes out of [1, 2^34]");
  if (path != HC_TUNE_BATCHED && path != HC_TUNE_SINGLE)
    return set_error(HC_ERR_ARG, "hc_tuner_calibrate: path must be HC_TUNE_BATCHED or HC_TUNE_SINGLE");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  uint8_t* y = nullptr;
  e = cudaMalloc(&y, text_bytes);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(calibration text)");
  Scratch sc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HC_OK;
  e = cudaMalloc(&sc.args, sizeof(SearchArgs));
  if (e == cudaSuccess) e = cudaMalloc(&sc.counter, (kMaxScanClasses + 1) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) rc = cuda_error(e, "hc_tuner_calibrate setup");
  const DeviceInfo& di = device_info(dev);
  for (size_t si = 0; si < nsigma && rc == HC_OK; ++si) {
    hc_tune_text_kernel<<<di.sm_count * 8, 256, 0, stream>>>(y, text_bytes, sigmas[si],
                                                             seed + 0x1000003ull * sigmas[si]);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = cuda_error(e, "hc_tune_text_kernel launch");
      break;
    }
    g_launches.fetch_add(1);
    for (size_t mi = 0; mi < nm && rc == HC_OK; ++mi)
      rc = calibrate_cell(t, sc, dev, y, text_bytes, sigmas[si], ms[mi], seed, path, stream, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(stream);
  cudaFree(y);
  return rc;
}

int hc_tuner_lookup(const hc_tuner* tp, double sigma, uint64_t m, hc_tune_entry* out) {
  clear_error();
  if (out == nullptr) return set_error(HC_ERR_ARG, "hc_tuner_lookup: out is NULL");
  const Tuner* t = nullptr;
  if (tp != nullptr && (t = as_tuner(tp)) == nullptr) return set_error(HC_ERR_ARG, "hc_tuner_lookup: invalid tuner");
  if (m < 1) return set_error(HC_ERR_ARG, "hc_tuner_lookup: m = 0");
  const QueryParams p = tuner_lookup(t, sigma, m);
  *out = hc_tune_entry{};
  out->sigma = static_cast<int>(std::lround(sigma));
  out->m = m;
  out->q = p.q;
  out->alpha = p.alpha;
  out->lane_bytes = p.lane_bytes;
  out->mode = p.mode;
  out->sentinel = p.sentinel;
  out->bitmap = p.bitmap;
  return HC_OK;
}

int hc_tuner_size(const hc_tuner* tp, size_t* count) {
  Tuner* t = as_tuner(tp);
  if (t == nullptr || count == nullptr) return set_error(HC_ERR_ARG, "hc_tuner_size: invalid argument");
  std::lock_guard<std::mutex> lock(t->mu);
  *count = t->cells.size();
  return HC_OK;
}

int hc_tuner_entry(const hc_tuner* tp, size_t i, hc_tune_entry* out) {
  Tuner* t = as_tuner(tp);
  if (t == nullptr || out == nullptr) return set_error(HC_ERR_ARG, "hc_tuner_entry: invalid argument");
  std::lock_guard<std::mutex> lock(t->mu);
  if (i >= t->cells.size()) return set_error(HC_ERR_ARG, "hc_tuner_entry: index out of range");
  *out = t->cells[i];
  return HC_OK;
}

int hc_tuner_save(const hc_tuner* tp, const char* path) {
  clear_error();
  Tuner* t = as_tuner(tp);
  if (t == nullptr || path == nullptr) return set_error(HC_ERR_ARG, "hc_tuner_save: invalid argument");
  FILE* f = std::fopen(path, "w");
  if (f == nullptr) return set_error(HC_ERR_STATE, std::string("hc_tuner_save: cannot open ") + path);
  std::lock_guard<std::mutex> lock(t->mu);
  std::fprintf(f, "# sigma m q alpha lane_bytes mode gbps sentinel bitmap\n");
  for (const auto& c : t->cells)
    std::fprintf(f, "%d %llu %d %d %d %d %.3f %d %d\n", c.sigma, static_cast<unsigned long long>(c.m), c.q, c.alpha,
                 c.lane_bytes, c.mode, c.gbps, c.sentinel, c.bitmap);
  const bool ok = std::fclose(f) == 0;
  return ok ? HC_OK : set_error(HC_ERR_STATE, "hc_tuner_save: write failed");
}

int hc_tuner_load(hc_tuner* tp, const char* path) {
  clear_error();
  Tuner* t = as_tuner(tp);
  if (t == nullptr || path == nullptr) return set_error(HC_ERR_ARG, "hc_tuner_load: invalid argument");
  FILE* f = std::fopen(path, "r");
  if (f == nullptr) return set_error(HC_ERR_STATE, std::string("hc_tuner_load: cannot open ") + path);
  std::vector<hc_tune_entry> got;
  char line[256];
  int lineno = 0, rc = HC_OK;
  while (std::fgets(line, sizeof line, f) != nullptr) {
    ++lineno;
    const char* s = line;
    while (*s == ' ' || *s == '\t') ++s;
    if (*s == '#' || *s == '\n' || *s == '\0') continue;
    hc_tune_entry c{};
    unsigned long long m = 0;
    // the last two columns (sentinel form, bitmap form) are optional: 0
    // when absent
    const int got_fields = std::sscanf(s, "%d %llu %d %d %d %d %lf %d %d", &c.sigma, &m, &c.q, &c.alpha,
                                       &c.lane_bytes, &c.mode, &c.gbps, &c.sentinel, &c.bitmap);
    if (got_fields < 7 || c.sentinel < 0 || c.sentinel > 1 || (c.sentinel == 1 && c.mode != HC_MODE_STAGED) ||
        c.bitmap < 0 || c.bitmap > 1 || (c.bitmap == 1 && c.mode != HC_MODE_DENSE) ||
        c.sigma < 1 || m < 1 || c.q < 1 || c.q > kMaxQ || static_cast<unsigned long long>(c.q) > m ||
        c.alpha < 1 || c.alpha > kMaxAlpha || c.lane_bytes < 0 || c.lane_bytes > 4096 ||
        (c.mode != HC_MODE_AUTO && c.mode != HC_MODE_STAGED && c.mode != HC_MODE_DIRECT &&
         !(c.mode == HC_MODE_DENSE && static_cast<unsigned long long>(c.q) == m))) {
      rc = set_error(HC_ERR_STATE, std::string("hc_tuner_load: malformed line ") + std::to_string(lineno));
      break;
    }
    c.m = m;
    got.push_back(c);
  }
  std::fclose(f);
  if (rc != HC_OK) return rc;
  std::lock_guard<std::mutex> lock(t->mu);
  for (const auto& c : got) put_cell(t, c);
  return HC_OK;
}

}  // extern "C"
