// zig_tune.cpp -- the autotuner's cache of chosen launch shapes: an
// in-process table keyed by (device name, SM count, dist, dtype), read from
// and written to JSON Lines files.  Host code only; the timing runs in
// zig_gen.cu.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "zig_internal.h"

namespace zig {
namespace {

typedef std::tuple<std::string, int, int, int> Key;  // device, sms, dist, dtype
std::mutex g_cache_mu;
std::map<Key, zig_tune_entry> g_cache;

const char* dist_name(int d) { return d == ZIG_EXP ? "exp" : "normal"; }
const char* dtype_name(int t) { return t == ZIG_F64 ? "f64" : "f32"; }

// Value of "key": in a one-line JSON object: a string (no escapes other
// than \" and \\) into str, or a number into num.  Returns false if absent.
bool field(const std::string& line, const char* key, std::string* str, double* num) {
  const std::string pat = std::string("\"") + key + "\"";
  size_t p = line.find(pat);
  if (p == std::string::npos) return false;
  p += pat.size();
  while (p < line.size() && (line[p] == ' ' || line[p] == '\t')) ++p;
  if (p >= line.size() || line[p] != ':') return false;
  ++p;
  while (p < line.size() && (line[p] == ' ' || line[p] == '\t')) ++p;
  if (p >= line.size()) return false;
  if (line[p] == '"') {
    if (!str) return false;
    str->clear();
    for (++p; p < line.size() && line[p] != '"'; ++p) {
      if (line[p] == '\\' && p + 1 < line.size()) ++p;
      str->push_back(line[p]);
    }
    return p < line.size();
  }
  if (!num) return false;
  char* end = nullptr;
  const double v = std::strtod(line.c_str() + p, &end);
  if (end == line.c_str() + p) return false;
  *num = v;
  return true;
}

std::string escaped(const std::string& s) {
  std::string o;
  for (char c : s) {
    if (c == '"' || c == '\\') o.push_back('\\');
    if ((unsigned char)c >= 0x20) o.push_back(c);
  }
  return o;
}

}  // namespace

void tune_cache_put(const char* device, int sms, int dist, int dtype, const zig_tune_entry& e) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  g_cache[Key(device, sms, dist, dtype)] = e;
}

bool tune_cache_get(const char* device, int sms, int dist, int dtype, zig_tune_entry* e) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_cache.find(Key(device, sms, dist, dtype));
  if (it == g_cache.end()) return false;
  *e = it->second;
  return true;
}

int tune_cache_load(const char* path) {
  if (!path) return ZIG_E_INVAL;
  FILE* f = std::fopen(path, "r");
  if (!f) return ZIG_E_INVAL;
  std::string line;
  int c;
  bool eof = false;
  while (!eof) {
    line.clear();
    while ((c = std::fgetc(f)) != EOF && c != '\n') line.push_back((char)c);
    eof = c == EOF;
    std::string dev, dist, dtype;
    double sms = 0, V = 0, R = 0, mb = 0, bps = 0, rate = 0;
    if (!field(line, "device", &dev, nullptr) || !field(line, "sms", nullptr, &sms) ||
        !field(line, "dist", &dist, nullptr) || !field(line, "dtype", &dtype, nullptr) ||
        !field(line, "V", nullptr, &V) || !field(line, "R", nullptr, &R) ||
        !field(line, "min_blocks", nullptr, &mb) || !field(line, "blocks_per_sm", nullptr, &bps))
      continue;
    field(line, "gsamples_s", nullptr, &rate);
    const int d = dist == "exp" ? ZIG_EXP : dist == "normal" ? ZIG_NORMAL : -1;
    const int t = dtype == "f32" ? ZIG_F32 : dtype == "f64" ? ZIG_F64 : -1;
    if (d < 0 || t < 0 || sms < 1 || bps < 0) continue;
    zig_tune_entry e{(int32_t)V, (int32_t)R, (int32_t)mb, (int32_t)bps, rate};
    if (!tune_shape_known(t, e)) continue;
    tune_cache_put(dev.c_str(), (int)sms, d, t, e);
  }
  std::fclose(f);
  return ZIG_OK;
}

int tune_cache_save(const char* path) {
  if (!path) return ZIG_E_INVAL;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return ZIG_E_CUDA;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (const auto& kv : g_cache) {
      const zig_tune_entry& e = kv.second;
      std::fprintf(f,
                   "{\"device\": \"%s\", \"sms\": %d, \"dist\": \"%s\", \"dtype\": \"%s\", "
                   "\"V\": %d, \"R\": %d, \"min_blocks\": %d, \"blocks_per_sm\": %d, "
                   "\"gsamples_s\": %.3f}\n",
                   escaped(std::get<0>(kv.first)).c_str(), std::get<1>(kv.first),
                   dist_name(std::get<2>(kv.first)), dtype_name(std::get<3>(kv.first)), e.V, e.R,
                   e.min_blocks, e.blocks_per_sm, e.gsamples_s);
    }
  }
  const bool ok = std::fclose(f) == 0;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return ZIG_E_CUDA;
  }
  return ZIG_OK;
}

}  // namespace zig

extern "C" {

zig_status zig_tune_save(const char* path) { return (zig_status)zig::tune_cache_save(path); }

zig_status zig_tune_load(const char* path) {
  const int st = zig::tune_cache_load(path);
  if (st == ZIG_OK) zig::tune_apply_loaded();
  return (zig_status)st;
}

}  // extern "C"
