// hc_batch_internal.h -- planning and launching of batched searches, shared
// by hc_batch_* (a planned table replayed by the caller), the autotuner
// (single-query batches timed on calibration texts) and the server (batches
// assembled from queued requests in stream-ordered memory).
//
// A plan is host data only: per query the launch arguments (SearchArgs), and
// for the whole batch the scan tiles (query, 8 records), the emit tiles
// (query, record group) and the sizes of the filter and workspace areas.
// plan_bind() writes the device addresses of those areas into the arguments;
// launch_batch() enqueues the three kernels of a batch.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "hc_internal.h"
#include "hc_kernels.cuh"

namespace hc {

struct BatchTile {
  uint32_t query;
  uint32_t first_record;
};

struct EmitTile {
  uint32_t query;
  uint32_t group;
};

struct BatchLayout {
  uint32_t f_bytes;     // shared memory for F (largest query)
  uint32_t x_bytes;     // shared memory for x (largest staged pattern)
  uint32_t ring_bytes;  // per-warp staging ring (largest query)
};

// Search parameters of one query: q and alpha of the filter, window starts
// per lane (0 = automatic) and scan mode (HC_MODE_AUTO, _STAGED, _DIRECT).
struct QueryParams {
  int q = 0, alpha = 0, lane_bytes = 0, mode = 0;
  int sentinel = 0;  // single searches in the staged mode: the sentinel form
  int bitmap = 0;    // single searches in the dense mode: the bitmap form
};

// Queries are grouped by the number of CTAs per SM their own shared-memory
// layout allows (filter, pattern and staging ring differ per query); each
// group runs as one persistent scan whose layout is the group's largest, so
// one query with a large filter or ring does not lower the occupancy of the
// whole batch.
constexpr int kMaxScanClasses = 4;

struct ScanClass {
  unsigned long long tile_begin = 0, ntiles = 0;  // its tiles: tiles[tile_begin ..)
  BatchLayout lay{};
  size_t smem = 0;  // dynamic shared memory of its scan launch
  int grid = 0;     // persistent grid of its scan launch
};

struct BatchPlan {
  std::vector<SearchArgs> args;
  std::vector<ScanClass> classes;  // set by plan_finish; tiles are sorted by class
  std::vector<QueryParams> params;
  std::vector<BatchTile> tiles;
  std::vector<EmitTile> etiles;
  std::vector<size_t> f_off;   // filter area offset of each query, in words
  std::vector<size_t> ws_off;  // workspace area offset of each query, in bytes
  size_t filter_words = 0;     // size of the filter area (16-byte multiple)
  size_t ws_bytes = 0;         // size of the workspace area (16-byte multiple)
  unsigned long long records = 0;
  BatchLayout lay{};
  size_t smem_pre = 0, smem_scan = 0, smem_emit = 0;
};

// Text bytes per record (one warp's share of a query) for a batch of
// `total_text` bytes on device dev: enough records to give every warp slot
// of the GPU (SMs x 16) work when the batch is small, at most 64 KiB each.
unsigned long long record_bytes_for(unsigned long long total_text, int dev);

// Appends query Q (index i, for messages) with parameters p to the plan, its
// text cut into records of about record_bytes (whole chunks, at least one).
// Checks pointers, alignment and parameter ranges; reads no device memory.
int plan_add_query(BatchPlan& plan, const hc_batch_query& Q, size_t i, const QueryParams& p,
                   unsigned long long record_bytes, const char* who);
// Scan classes (tiles sorted by class, each class's layout, shared memory
// and grid) and the emit layout; HC_ERR_ARG when a query's filter and
// staging buffers do not fit in one CTA.
int plan_finish(BatchPlan& plan, int dev, const char* who);
// Writes the device addresses of the filter area (filter_words words) and
// the workspace area (ws_bytes bytes, 16-byte aligned) into the arguments.
void plan_bind(BatchPlan& plan, uint32_t* d_filters, uint8_t* d_ws);

// Everything one run of a planned batch needs on the device.
struct BatchLaunch {
  const SearchArgs* args = nullptr;  // nq arguments
  const BatchTile* tiles = nullptr;  // sorted by scan class
  const EmitTile* etiles = nullptr;
  unsigned long long* counters = nullptr;  // kMaxScanClasses work counters (reset by the run)
  size_t nq = 0;
  unsigned long long netiles = 0;
  ScanClass classes[kMaxScanClasses];
  int nclasses = 0;
  size_t smem_pre = 0, smem_emit = 0;
};

// Persistent grid of each scan class on device dev (SMs x resident CTAs, at
// most one CTA per tile).
int batch_grids(BatchPlan& plan, int dev);

// The launch description of a plan whose tables are at the given device
// addresses (counters: kMaxScanClasses of them).
BatchLaunch make_launch(const BatchPlan& plan, const SearchArgs* args, const BatchTile* tiles,
                        const EmitTile* etiles, unsigned long long* counters);
// Enqueues preprocessing, scan and emit on `stream`; allocates nothing and
// is graph-capturable.  Counts its launches.
int launch_batch(const BatchLaunch& L, cudaStream_t stream);

// Effective alphabet size of each text, 1 / sum(p_c^2) over the byte
// frequencies of a sample (all of a text up to 64 KiB, else 16 evenly spaced
// pieces of 4 KiB); 0 for an empty text.  Synchronous.
int estimate_sigma(const uint8_t* const* y_dev, const uint64_t* n, size_t count,
                   std::vector<double>* sigma, cudaStream_t stream);

// Autotuner lookup (a NULL tuner gives the paper's table).
struct Tuner;
Tuner* as_tuner(const hc_tuner* t);
QueryParams tuner_lookup(const Tuner* t, double sigma, uint64_t m);

}  // namespace hc
