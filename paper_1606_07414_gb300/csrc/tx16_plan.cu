// Batch plans (tx16_plan_*): one persistent, fused launch per zonal class over
// a batch of images of uneven sizes, driven by a device-side work list.
//
// The work list is the table of per-image descriptors (ImgParam) in device
// memory, grouped by zonal class, plus one tile counter per class.  CTAs of
// the work-list kernel claim chunks of tiles from their class's counter (for
// classes up to 8 kept columns without levels, warps of the one-block-per-
// thread kernel claim warp tiles of 32 blocks), so
// images with more kept coefficients (dearer columns) and uneven sizes balance
// across the SMs without any host-side partitioning.  A run is
//   memset(sse), memset(counters), one launch per class (+ the general kernel
//   for 16-bit planes or steps below the fused kernel's range),
// and can be captured once into a CUDA graph and replayed.  The autotuner
// times the schedule parameters (resident CTAs per SM, tiles per claim) of
// each class on the plan's own data and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tx16_internal.h"

namespace tx16 {
ImgParam make_param(const tx16_image& in, const tx16_image* out, const tx16_qparams& qp, int64_t blk0);
bool valid_qparams(const tx16_qparams& qp);
}  // namespace tx16

using namespace tx16;

namespace {

struct ClassRun {
  int zone;        // 0..5 fused zone class, -1: general kernel (by value, host table)
  int first;       // first descriptor of the run in the table
  int count;       // descriptors in the run
  int ntiles;      // tiles of the run (16 blocks, pair kernel)
  int ctas_per_sm; // 0: as many as fit
  int chunk;       // tiles per claim
  // classes the one-block-per-thread kernel can take when no levels are
  // asked: its own table (tile0 in warp tiles of 32 blocks) and schedule
  bool bt;  // the mapping a run without levels uses: one block per thread (else the pair kernel)
  int bt_ntiles, bt_ctas_per_sm, bt_chunk;
  int bt_variant;  // compiled configuration of that kernel (0: the default)
  bool bt_ok;      // the one-block-per-thread kernel takes this class
};

}  // namespace

struct tx16_plan {
  int device = 0;
  int n = 0;
  bool has_dst = false;
  std::vector<ImgParam> table;  // grouped by run; tile0 relative to the run
  std::vector<ImgParam> bt_table;  // the same descriptors, tile0 in warp tiles
  std::vector<ClassRun> runs;
  ImgParam* d_table = nullptr;
  ImgParam* d_bt_table = nullptr;
  unsigned* d_counters = nullptr;
  // graph of one run, keyed by the output pointers it was captured with
  cudaGraphExec_t graph = nullptr;
  uint64_t* graph_sse = nullptr;
  int32_t* graph_levels = nullptr;
  cudaStream_t capture_stream = nullptr;
};

namespace {

int fused_tiles(int nblk) { return (nblk + 15) / 16; }

tx16_status run_plan(tx16_plan* p, uint64_t* sse, int32_t* levels, cudaStream_t st) {
  if (sse != nullptr && cudaMemsetAsync(sse, 0, sizeof(uint64_t) * size_t(p->n), st) != cudaSuccess)
    return TX16_ECUDA;
  if (!p->runs.empty() &&
      cudaMemsetAsync(p->d_counters, 0, sizeof(unsigned) * p->runs.size(), st) != cudaSuccess)
    return TX16_ECUDA;
  unsigned long long* s64 = reinterpret_cast<unsigned long long*>(sse);
  for (size_t i = 0; i < p->runs.size(); ++i) {
    const ClassRun& r = p->runs[i];
    tx16_status s;
    if (r.zone >= 0 && r.bt && levels == nullptr) {
      s = launch_fused_bt_list(r.zone, r.bt_variant, p->has_dst, p->d_bt_table + r.first, r.count, r.bt_ntiles,
                               p->d_counters + i, r.bt_chunk, r.bt_ctas_per_sm, s64, st);
    } else if (r.zone >= 0) {
      s = launch_fused_list(r.zone, levels != nullptr, p->has_dst, p->d_table + r.first, r.count, r.ntiles,
                            p->d_counters + i, r.chunk, r.ctas_per_sm, s64, levels, st);
    } else {
      // general kernel: descriptors by value, SSE indices = the images' own
      // (one launch per image keeps out_index and the launch index equal)
      s = TX16_OK;
      for (int j = 0; j < r.count && s == TX16_OK; ++j) {
        ImgParam q = p->table[r.first + j];
        unsigned long long* sj = s64 ? s64 + q.out_index : nullptr;
        s = launch_blocks(kOpCodec, (q.flags & 0xff) == 8 ? 1 : 2, &q, 1, sj, levels, st);
      }
    }
    if (s != TX16_OK) return s;
  }
  return TX16_OK;
}

}  // namespace

extern "C" {

tx16_status tx16_plan_create(const tx16_image* in, const tx16_image* out, int32_t n, const tx16_qparams* qp,
                             tx16_plan** plan) {
  TX16_TRACE("tx16_plan_create");
  if (plan == nullptr) return TX16_EINVAL;
  *plan = nullptr;
  if (n <= 0 || in == nullptr || qp == nullptr) return TX16_EINVAL;
  std::vector<ImgParam> params(n);
  std::vector<int> cls(n);
  int64_t blk0 = 0;
  for (int i = 0; i < n; ++i) {
    if (!valid_image(in[i]) || !valid_qparams(qp[i])) return TX16_EINVAL;
    if (out != nullptr && (!valid_image(out[i]) || out[i].width != in[i].width ||
                           out[i].height != in[i].height || out[i].bits != in[i].bits))
      return TX16_EINVAL;
    params[i] = make_param(in[i], out ? &out[i] : nullptr, qp[i], blk0);
    params[i].out_index = i;
    blk0 += params[i].nblk;
    const bool fast = in[i].bits == 8 && (qp[i].q <= 0.f || qp[i].q >= kFusedMinQ);
    cls[i] = fast ? fused_zone_class(&params[i], 1) : -1;
  }
  tx16_plan* p = new tx16_plan();
  cudaGetDevice(&p->device);
  p->n = n;
  p->has_dst = out != nullptr;
  for (int c = -1; c <= 5; ++c) {
    const bool bt_ok = c >= 0 && fused_bt_supports(c, false);
    ClassRun r{c, int(p->table.size()), 0, 0, 0, 1, bt_ok, 0, 0, 1, 0, bt_ok};
    for (int i = 0; i < n; ++i) {
      if (cls[i] != c) continue;
      ImgParam q = params[i];
      q.tile0 = r.ntiles;
      r.ntiles += fused_tiles(q.nblk);
      p->table.push_back(q);
      q.tile0 = r.bt_ntiles;
      r.bt_ntiles += bt_warp_tiles(q.nblk);
      p->bt_table.push_back(q);
      ++r.count;
    }
    if (r.count == 0) continue;
    // default schedules: all resident CTAs, claims sized for ~8 claims per
    // CTA (pair kernel) or per warp of 4-warp CTAs (one block per thread)
    if (c >= 0) {
      const int ctas = fused_list_max_ctas(c, false, p->has_dst) * device_sm_count();
      r.chunk = std::max(1, std::min(16, r.ntiles / std::max(1, ctas * 8)));
    }
    if (r.bt) {
      const int warps = fused_bt_list_max_ctas(c, 0, p->has_dst) * device_sm_count() * fused_bt_warps_per_cta(c);
      r.bt_chunk = std::max(1, std::min(16, r.bt_ntiles / std::max(1, warps * 8)));
    }
    p->runs.push_back(r);
  }
  if (cudaMalloc(&p->d_table, sizeof(ImgParam) * p->table.size()) != cudaSuccess ||
      cudaMalloc(&p->d_bt_table, sizeof(ImgParam) * p->bt_table.size()) != cudaSuccess ||
      cudaMalloc(&p->d_counters, sizeof(unsigned) * std::max<size_t>(1, p->runs.size())) != cudaSuccess) {
    tx16_plan_destroy(p);
    return TX16_ENOMEM;
  }
  if (cudaMemcpy(p->d_table, p->table.data(), sizeof(ImgParam) * p->table.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(p->d_bt_table, p->bt_table.data(), sizeof(ImgParam) * p->bt_table.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    tx16_plan_destroy(p);
    return TX16_ECUDA;
  }
  *plan = p;
  return TX16_OK;
}

tx16_status tx16_plan_run(tx16_plan* plan, uint64_t* sse, int32_t* levels, void* stream) {
  TX16_TRACE("tx16_plan_run");
  if (plan == nullptr) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(sse) & 7u) != 0 || (reinterpret_cast<uintptr_t>(levels) & 15u) != 0)
    return TX16_EINVAL;
  return run_plan(plan, sse, levels, static_cast<cudaStream_t>(stream));
}

tx16_status tx16_plan_run_graph(tx16_plan* plan, uint64_t* sse, int32_t* levels, void* stream) {
  TX16_TRACE("tx16_plan_run_graph");
  if (plan == nullptr) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(sse) & 7u) != 0 || (reinterpret_cast<uintptr_t>(levels) & 15u) != 0)
    return TX16_EINVAL;
  if (plan->graph == nullptr || plan->graph_sse != sse || plan->graph_levels != levels) {
    // occupancy queries happen on first use of a kernel: do them before capture
    for (const ClassRun& r : plan->runs) {
      if (r.zone >= 0) fused_list_max_ctas(r.zone, levels != nullptr, plan->has_dst);
      if (r.bt) fused_bt_list_max_ctas(r.zone, r.bt_variant, plan->has_dst);
    }
    if (plan->graph != nullptr) {
      cudaGraphExecDestroy(plan->graph);
      plan->graph = nullptr;
    }
    if (plan->capture_stream == nullptr &&
        cudaStreamCreateWithFlags(&plan->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
      return TX16_ECUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(plan->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return TX16_ECUDA;
    const tx16_status s = run_plan(plan, sse, levels, plan->capture_stream);
    const cudaError_t e = cudaStreamEndCapture(plan->capture_stream, &g);
    if (s != TX16_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return s != TX16_OK ? s : TX16_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&plan->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      plan->graph = nullptr;
      return TX16_ECUDA;
    }
    plan->graph_sse = sse;
    plan->graph_levels = levels;
  }
  return cudaGraphLaunch(plan->graph, static_cast<cudaStream_t>(stream)) == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

tx16_status tx16_plan_autotune(tx16_plan* plan, const char* cache_path, void* stream) {
  TX16_TRACE("tx16_plan_autotune");
  if (plan == nullptr) return TX16_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, plan->device) != cudaSuccess) return TX16_ECUDA;
  // cache: one line per class, "device|zone|dst|tiles_bucket[|bt] ctas chunk variant" (variant -1:
  // the pair kernel)
  std::vector<std::string> cache;
  if (cache_path != nullptr) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[512];
      while (std::fgets(line, sizeof line, f)) cache.emplace_back(line);
      std::fclose(f);
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TX16_ECUDA;
  bool changed = false;
  for (size_t i = 0; i < plan->runs.size(); ++i) {
    ClassRun& r = plan->runs[i];
    if (r.zone < 0) continue;
    const int bucket = int(std::log2(double(std::max(1, r.ntiles))));
    std::string dev(prop.name);
    std::replace(dev.begin(), dev.end(), ' ', '_');  // keys are single words in the cache file
    char key[320];
    // the schedule tuned is that of the kernel a run without levels uses
    std::snprintf(key, sizeof key, "%s|%d|%d|%d%s", dev.c_str(), r.zone, int(plan->has_dst), bucket,
                  r.bt_ok ? "|bt" : "");
    const int nvar = r.bt_ok ? fused_bt_variants(r.zone) : 0;
    // apply a schedule: var >= 0 a configuration of the one-block-per-thread
    // kernel, -1 the pair kernel (two blocks per float2 pair, 16 threads per
    // pair of blocks: the other mapping of rows and columns to lanes)
    auto apply = [&](int var, int ctas, int chunk) {
      r.bt = var >= 0;
      if (r.bt) {
        r.bt_variant = var;
        r.bt_ctas_per_sm = ctas;
        r.bt_chunk = chunk;
      } else {
        r.ctas_per_sm = ctas;
        r.chunk = chunk;
      }
    };
    bool hit = false;
    for (const std::string& c : cache) {
      int ctas = 0, chunk = 0, var = -1;
      char k2[320];
      const int got = std::sscanf(c.c_str(), "%319s %d %d %d", k2, &ctas, &chunk, &var);
      if (got < 3 || std::string(k2) != key) continue;
      if (!r.bt_ok) var = -1;
      if (var >= nvar) continue;
      apply(var, ctas, chunk);
      hit = true;
    }
    if (hit) continue;
    // candidates: the pair kernel and each compiled configuration of the
    // one-block-per-thread kernel (warps per CTA, parked column pairs, input
    // stages), and for each its resident CTAs per SM (the most that fit and
    // up to 4 fewer) and tiles per claim
    float best = 1e30f;
    int best_ctas = 0, best_chunk = 1, best_var = -1;
    const int chunks[] = {0, 1, 2, 4, 8, 16};  // 0: a static contiguous run per CTA (one block per thread)
    for (int var = -1; var < nvar; ++var) {
      const bool use_bt = var >= 0;
      const int maxc = use_bt ? fused_bt_list_max_ctas(r.zone, var, plan->has_dst)
                              : fused_list_max_ctas(r.zone, false, plan->has_dst);
      if (maxc <= 0) continue;
      int warps = 1, park = 0, stages = 1;
      if (use_bt) fused_bt_variant_info(r.zone, var, &warps, &park, &stages);
      const int claimers_per_cta = use_bt ? warps : 1;  // warps of a one-block-per-thread CTA claim separately
      const int tiles = use_bt ? r.bt_ntiles : r.ntiles;
      for (int ctas = maxc; ctas >= 1 && ctas >= maxc - 4; --ctas) {
        for (int chunk : chunks) {
          if (chunk == 0 && !use_bt) continue;
          if (chunk > std::max(1, tiles / (ctas * claimers_per_cta * device_sm_count()))) continue;
          float ms = 0.f;
          for (int rep = 0; rep < 3; ++rep) {
            if (cudaMemsetAsync(plan->d_counters + i, 0, sizeof(unsigned), st) != cudaSuccess) return TX16_ECUDA;
            cudaEventRecord(e0, st);
            const tx16_status ls =
                use_bt ? launch_fused_bt_list(r.zone, var, plan->has_dst, plan->d_bt_table + r.first, r.count,
                                              r.bt_ntiles, plan->d_counters + i, chunk, ctas, nullptr, st)
                       : launch_fused_list(r.zone, false, plan->has_dst, plan->d_table + r.first, r.count, r.ntiles,
                                           plan->d_counters + i, chunk, ctas, nullptr, nullptr, st);
            if (ls != TX16_OK) return TX16_ECUDA;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return TX16_ECUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t;  // first repetition warms up
          }
          if (ms < best) {
            best = ms;
            best_ctas = ctas;
            best_chunk = chunk;
            best_var = var;
          }
        }
      }
    }
    if (best == 1e30f) continue;  // nothing could run: keep the defaults
    apply(best_var, best_ctas, best_chunk);
    char line[400];
    std::snprintf(line, sizeof line, "%s %d %d %d\n", key, best_ctas, best_chunk, best_var);
    cache.emplace_back(line);
    changed = true;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (plan->graph != nullptr) {  // schedule changed: re-capture on next graph run
    cudaGraphExecDestroy(plan->graph);
    plan->graph = nullptr;
  }
  if (changed && cache_path != nullptr) {
    if (FILE* f = std::fopen(cache_path, "w")) {
      for (const std::string& c : cache) std::fputs(c.c_str(), f);
      std::fclose(f);
    }
  }
  return TX16_OK;
}

tx16_status tx16_plan_info(const tx16_plan* plan, int32_t* runs, int32_t* zone, int32_t* tiles, int32_t* ctas_per_sm,
                           int32_t* chunk, int32_t max_runs) {
  if (plan == nullptr || runs == nullptr) return TX16_EINVAL;
  *runs = int32_t(plan->runs.size());
  for (int i = 0; i < *runs && i < max_runs; ++i) {
    // the schedule of the kernel a run without levels uses
    const ClassRun& r = plan->runs[i];
    if (zone) zone[i] = r.zone;
    if (tiles) tiles[i] = r.bt ? r.bt_ntiles : r.ntiles;
    if (ctas_per_sm) ctas_per_sm[i] = r.bt ? r.bt_ctas_per_sm : r.ctas_per_sm;
    if (chunk) chunk[i] = r.bt ? r.bt_chunk : r.chunk;
  }
  return TX16_OK;
}

tx16_status tx16_plan_variant(const tx16_plan* plan, int32_t run, int32_t* variant, int32_t* warps_per_cta,
                              int32_t* parked_pairs, int32_t* stages) {
  if (plan == nullptr || run < 0 || run >= int32_t(plan->runs.size())) return TX16_EINVAL;
  const ClassRun& r = plan->runs[run];
  int w = 0, pk = 0, sg = 0;
  if (r.bt) fused_bt_variant_info(r.zone, r.bt_variant, &w, &pk, &sg);
  if (variant) *variant = r.bt ? r.bt_variant : -1;
  if (warps_per_cta) *warps_per_cta = w;
  if (parked_pairs) *parked_pairs = pk;
  if (stages) *stages = sg;
  return TX16_OK;
}

tx16_status tx16_plan_set_schedule(tx16_plan* plan, int32_t run, int32_t variant, int32_t ctas_per_sm,
                                   int32_t chunk) {
  if (plan == nullptr || run < 0 || run >= int32_t(plan->runs.size()) || ctas_per_sm < 0 || chunk < 0)
    return TX16_EINVAL;
  ClassRun& r = plan->runs[run];
  if (r.zone < 0) return TX16_EINVAL;  // the general kernel has no schedule
  if (r.bt_ok && variant >= 0) {
    if (variant >= fused_bt_variants(r.zone)) return TX16_EINVAL;
    r.bt = true;
    r.bt_variant = variant;
    r.bt_ctas_per_sm = ctas_per_sm;
    r.bt_chunk = chunk;
  } else {
    if (variant != -1 && !(variant == 0 && !r.bt_ok)) return TX16_EINVAL;  // the pair kernel
    if (chunk < 1) return TX16_EINVAL;  // claims only
    r.bt = false;
    r.ctas_per_sm = ctas_per_sm;
    r.chunk = chunk;
  }
  if (plan->graph != nullptr) {  // schedule changed: re-capture on next graph run
    cudaGraphExecDestroy(plan->graph);
    plan->graph = nullptr;
  }
  return TX16_OK;
}

void tx16_plan_destroy(tx16_plan* plan) {
  if (plan == nullptr) return;
  if (plan->graph) cudaGraphExecDestroy(plan->graph);
  if (plan->capture_stream) cudaStreamDestroy(plan->capture_stream);
  if (plan->d_table) cudaFree(plan->d_table);
  if (plan->d_bt_table) cudaFree(plan->d_bt_table);
  if (plan->d_counters) cudaFree(plan->d_counters);
  delete plan;
}

}  // extern "C"
