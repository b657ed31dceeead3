// Tuned choices of the radix pass and of the batch wave size, per GPU and
// size class, kept in memory and optionally in a JSON cache file.
//
// A choice is keyed by (GPU name, kind, size class): kind 0 is a single
// table, kind 1 a batch; the size class is floor(log2(rows)) of the table,
// or of the mean selection of a batch.  ringo_tune_table and
// ringo_batch_autotune measure the candidates on the caller's own data and
// record the fastest; later conversions of the same class use it.  With a
// cache file set (ringo_tune_set_cache) the choices survive the process: the
// file is read when it is set and rewritten after every new choice.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <chrono>
#include <fstream>
#include <map>
#include <mutex>
#include <regex>
#include <sstream>
#include <string>
#include <tuple>

#include "../../include/ringo.h"
#include "host_util.h"
#include "ringo_internal.cuh"

namespace ringo {
namespace {

struct TuneEntry {
  SweepOpts opts;
  int64_t wave_rows = 0;
  double ms = 0;
  int out_passes = 0, in_passes = 0;
};
using TuneKey = std::tuple<std::string, int, int>;  // gpu, kind, size class

std::mutex g_mu;
std::map<TuneKey, TuneEntry> g_entries;
std::string g_path;
bool g_forced = false;
SweepOpts g_force;

int size_class(uint64_t rows) {
  int c = 0;
  while ((rows >> c) > 1) ++c;
  return c;
}

std::string gpu_name() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return std::string();
  }
  return std::string(p.name);
}

std::string json_escape(const std::string& x) {
  std::string o;
  for (char c : x) {
    if (c == '"' || c == '\\') o += '\\';
    if ((unsigned char)c >= 0x20) o += c;
  }
  return o;
}

// Writes every entry (caller holds g_mu).
void save_locked() {
  if (g_path.empty()) return;
  std::ostringstream o;
  o << "{\"version\": 1, \"entries\": [\n";
  bool first = true;
  for (const auto& kv : g_entries) {
    const TuneEntry& e = kv.second;
    o << (first ? "" : ",\n") << " {\"gpu\": \"" << json_escape(std::get<0>(kv.first))
      << "\", \"kind\": " << std::get<1>(kv.first) << ", \"size_class\": " << std::get<2>(kv.first)
      << ", \"rank_method\": " << e.opts.rank_method << ", \"prefetch_waves\": "
      << e.opts.prefetch_waves << ", \"in_digit_bits\": " << e.opts.in_digit_bits
      << ", \"wave_rows\": " << e.wave_rows << ", \"ms\": " << e.ms
      << ", \"out_passes\": " << e.out_passes << ", \"in_passes\": " << e.in_passes << "}";
    first = false;
  }
  o << "\n]}\n";
  const std::string tmp = g_path + ".tmp";
  {
    std::ofstream f(tmp, std::ios::trunc);
    if (!f) return;
    f << o.str();
  }
  std::rename(tmp.c_str(), g_path.c_str());
}

// Reads the entries of a cache file written by save_locked (caller holds
// g_mu); fields it does not know are ignored.  Returns false if the file
// exists but is not a cache file.
bool load_locked(const std::string& path) {
  std::ifstream f(path);
  if (!f) return true;  // no file yet
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string text = ss.str();
  if (text.find("\"entries\"") == std::string::npos) return false;
  const std::regex obj("\\{[^{}]*\\}");
  const std::regex num_field("\"([a-z_]+)\"\\s*:\\s*(-?[0-9.eE+]+)");
  const std::regex gpu_field("\"gpu\"\\s*:\\s*\"((?:[^\"\\\\]|\\\\.)*)\"");
  for (auto it = std::sregex_iterator(text.begin(), text.end(), obj); it != std::sregex_iterator();
       ++it) {
    const std::string o = it->str();
    std::smatch g;
    if (!std::regex_search(o, g, gpu_field)) continue;
    std::string gpu;
    for (size_t i = 0; i < g[1].str().size(); ++i) {
      const char c = g[1].str()[i];
      if (c == '\\' && i + 1 < g[1].str().size()) continue;
      gpu += c;
    }
    std::map<std::string, double> v;
    for (auto jt = std::sregex_iterator(o.begin(), o.end(), num_field); jt != std::sregex_iterator();
         ++jt)
      v[(*jt)[1].str()] = std::stod((*jt)[2].str());
    if (!v.count("kind") || !v.count("size_class")) continue;
    TuneEntry e;
    e.opts.rank_method = v.count("rank_method") ? (int)v["rank_method"] : 0;
    e.opts.prefetch_waves = v.count("prefetch_waves") ? (int)v["prefetch_waves"] : 1;
    e.opts.in_digit_bits = v.count("in_digit_bits") ? (int)v["in_digit_bits"] : 8;
    if (e.opts.rank_method < 0 || e.opts.rank_method > 2) e.opts.rank_method = 0;
    if (e.opts.prefetch_waves < 0 || e.opts.prefetch_waves > 2) e.opts.prefetch_waves = 1;
    if (e.opts.in_digit_bits != 9) e.opts.in_digit_bits = 8;
    e.wave_rows = v.count("wave_rows") ? (int64_t)v["wave_rows"] : 0;
    e.ms = v.count("ms") ? v["ms"] : 0;
    e.out_passes = v.count("out_passes") ? (int)v["out_passes"] : 0;
    e.in_passes = v.count("in_passes") ? (int)v["in_passes"] : 0;
    g_entries[TuneKey(gpu, (int)v["kind"], (int)v["size_class"])] = e;
  }
  return true;
}

bool valid_opts(const ringo_sort_opts* o) {
  return o && o->rank_method >= 0 && o->rank_method <= 2 && o->prefetch_waves >= 0 &&
         o->prefetch_waves <= 2 && o->wave_rows >= 0 &&
         (o->in_digit_bits == 0 || o->in_digit_bits == 8 || o->in_digit_bits == 9);
}

}  // namespace

ForcedOptsGuard::ForcedOptsGuard() {
  std::lock_guard<std::mutex> lk(g_mu);
  was = g_forced;
  saved = g_force;
}
ForcedOptsGuard::~ForcedOptsGuard() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_forced = was;
  g_force = saved;
}

SweepOpts sort_opts_for(int kind, uint64_t rows) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_forced) return g_force;
  if (g_entries.empty()) return SweepOpts{};
  auto it = g_entries.find(TuneKey(gpu_name(), kind, size_class(rows)));
  return it == g_entries.end() ? SweepOpts{} : it->second.opts;
}

int64_t tuned_wave_rows(uint64_t rows_per_pred) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_entries.empty()) return 0;
  auto it = g_entries.find(TuneKey(gpu_name(), 1, size_class(rows_per_pred)));
  return it == g_entries.end() ? 0 : it->second.wave_rows;
}

void record_tuned(int kind, uint64_t rows, const SweepOpts& o, int64_t wave_rows, double ms,
                  int out_passes, int in_passes) {
  const std::string gpu = gpu_name();
  std::lock_guard<std::mutex> lk(g_mu);
  TuneEntry e;
  e.opts = o;
  e.wave_rows = wave_rows;
  e.ms = ms;
  e.out_passes = out_passes;
  e.in_passes = in_passes;
  g_entries[TuneKey(gpu, kind, size_class(rows))] = e;
  save_locked();
}

}  // namespace ringo

using namespace ringo;

extern "C" {

int ringo_sort_opts_force(const ringo_sort_opts* opts) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!opts) {
    g_forced = false;
    return RINGO_OK;
  }
  if (!valid_opts(opts)) {
    set_error("ringo_sort_opts_force: rank_method outside 0..2, prefetch_waves outside 0..2, "
              "in_digit_bits not 0, 8 or 9, or wave_rows < 0");
    return RINGO_EINVAL;
  }
  g_force.rank_method = opts->rank_method;
  g_force.prefetch_waves = opts->prefetch_waves;
  g_force.in_digit_bits = opts->in_digit_bits == 9 ? 9 : 8;
  g_forced = true;
  return RINGO_OK;
}

int ringo_tune_set_cache(const char* path) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!path || !*path) {
    g_path.clear();
    return RINGO_OK;
  }
  if (!load_locked(path)) {
    set_error(std::string("ringo_tune_set_cache: not a tuning cache file: ") + path);
    return RINGO_EINVAL;
  }
  g_path = path;
  save_locked();
  return RINGO_OK;
}

int ringo_tune_lookup(int32_t kind, int64_t rows, ringo_sort_opts* opts, int32_t* found) {
  if (!opts || !found || (kind != 0 && kind != 1) || rows < 0) return RINGO_EINVAL;
  const std::string gpu = gpu_name();
  if (gpu.empty()) {
    set_error("ringo_tune_lookup: no usable current device");
    return RINGO_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_entries.find(TuneKey(gpu, kind, size_class((uint64_t)rows)));
  *found = it != g_entries.end() ? 1 : 0;
  const TuneEntry e = *found ? it->second : TuneEntry{};
  opts->rank_method = e.opts.rank_method;
  opts->prefetch_waves = e.opts.prefetch_waves;
  opts->wave_rows = e.wave_rows;
  opts->in_digit_bits = e.opts.in_digit_bits;
  return RINGO_OK;
}

int ringo_tune_table(const int32_t* src, const int32_t* dst, int64_t nrows, void* stream,
                     ringo_sort_opts* best, double* best_ms) {
  if (!best || nrows <= 0 || !src || !dst) {
    set_error("ringo_tune_table: NULL pointer or nrows <= 0");
    return RINGO_EINVAL;
  }
  SweepOpts best_o;
  ringo_graph_info info{};
  int rc = RINGO_OK;
  double best_t = 1e300;
  {
    const ForcedOptsGuard keep;  // candidates are forced one after another
    const auto measure = [&](const SweepOpts& so) {
      const ringo_sort_opts o{so.rank_method, so.prefetch_waves, 0, so.in_digit_bits, 0};
      ringo_sort_opts_force(&o);
      double t = 1e300;
      for (int rep = 0; rep < 3 && rc == RINGO_OK; ++rep) {  // the first run warms up
        cudaStreamSynchronize((cudaStream_t)stream);
        const auto t0 = std::chrono::steady_clock::now();
        ringo_graph* g = nullptr;
        rc = ringo_table_to_graph(src, dst, nrows, stream, &g);
        const double ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                .count();
        if (g) {
          ringo_graph_get_info(g, &info);
          ringo_graph_free(g);
        }
        if (rep > 0 && ms < t) t = ms;
      }
      if (rc == RINGO_OK && t < best_t) {
        best_t = t;
        best_o = so;
      }
    };
    for_each_candidate(measure, [&] { return best_o; }, [&] { return rc == RINGO_OK; });
  }
  if (rc != RINGO_OK) return rc;
  record_tuned(0, (uint64_t)nrows, best_o, 0, best_t, info.out_sort_passes, info.in_sort_passes);
  best->rank_method = best_o.rank_method;
  best->prefetch_waves = best_o.prefetch_waves;
  best->wave_rows = 0;
  best->in_digit_bits = best_o.in_digit_bits;
  if (best_ms) *best_ms = best_t;
  return RINGO_OK;
}

}  // extern "C"
