// A file cache for cb_autotune: the settings it chose, stored under a key
// that names the GPU and the shape of the handle's degree distribution, so a
// later handle of the same workload family on the same kind of GPU takes
// them without spending super steps on tuning (the tuner's result depends on
// the trade sizes, which the degree distribution fixes, and on the GPU).
//
// The key: the device name and SM count, floor(log2 n), floor(log2 graphs),
// and the share of directed entries (deg summed) of the nodes whose degree
// has bit length b, for b = 0..32, in 64ths (rounded).  Two graphs drawn
// from the same degree law at the same size share it.
//
// The file is JSON of this form, one object per key:
//   {"version": 1, "entries": [
//     {"key": "...", "tile_max": 32, "block_max": 2048, "smem_max": 2048,
//      "inorder_threads": 256, "retry_passes": 2}, ...]}
// It is written whole to a temporary file beside it, then renamed over it.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "cb_internal.cuh"

namespace cb {
namespace {

constexpr int kBits = 33;   // bit lengths of a degree (0 for degree 0)
constexpr int kTuneVals = 5;
const char* const kTuneNames[kTuneVals] = {"tile_max", "block_max", "smem_max", "inorder_threads", "retry_passes"};

// Directed entries (degrees summed) per degree bit length: shared-memory
// atomics, then one global atomic per bucket and block.
__global__ void k_degree_bits(int64_t n, const int64_t* __restrict__ rp, unsigned long long* __restrict__ out) {
  __shared__ unsigned long long ent[kBits];
  for (int i = threadIdx.x; i < kBits; i += blockDim.x) ent[i] = 0;
  __syncthreads();
  for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < n;
       x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t d = rp[x + 1] - rp[x];
    const int b = d > 0 ? 64 - __clzll(static_cast<unsigned long long>(d)) : 0;
    atomicAdd(&ent[b < kBits ? b : kBits - 1], static_cast<unsigned long long>(d));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kBits; i += blockDim.x)
    if (ent[i]) atomicAdd(out + i, ent[i]);
}

int floor_log2(int64_t v) {
  int b = -1;
  while (v > 0) {
    v >>= 1;
    ++b;
  }
  return b;
}

// The object of `key` in the file's text: [begin, end) of its braces, or
// begin = npos.
void find_entry(const std::string& text, const std::string& key, size_t* begin, size_t* end) {
  *begin = std::string::npos;
  const std::string needle = "\"key\": \"" + key + "\"";
  size_t at = 0;
  while ((at = text.find(needle, at)) != std::string::npos) {
    const size_t b = text.rfind('{', at);
    const size_t e = text.find('}', at);
    if (b != std::string::npos && e != std::string::npos) {
      *begin = b;
      *end = e + 1;
      return;
    }
    at += needle.size();
  }
}

bool read_file(const char* path, std::string* text, bool* exists) {
  *exists = false;
  FILE* f = std::fopen(path, "rb");
  if (!f) return true;   // no file yet: an empty cache
  *exists = true;
  char buf[4096];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) text->append(buf, k);
  const bool ok = !std::ferror(f);
  std::fclose(f);
  return ok;
}

bool parse_entry(const std::string& obj, int64_t* vals) {
  for (int i = 0; i < kTuneVals; ++i) {
    const std::string name = std::string("\"") + kTuneNames[i] + "\":";
    const size_t at = obj.find(name);
    if (at == std::string::npos) return false;
    const char* p = obj.c_str() + at + name.size();
    char* endp = nullptr;
    vals[i] = std::strtoll(p, &endp, 10);
    if (endp == p) return false;
  }
  return true;
}

std::string format_entry(const std::string& key, const int64_t* vals) {
  std::string s = "    {\"key\": \"" + key + "\"";
  for (int i = 0; i < kTuneVals; ++i) s += std::string(", \"") + kTuneNames[i] + "\": " + std::to_string(vals[i]);
  return s + "}";
}

bool valid_key(const char* key) {
  for (const char* p = key; *p; ++p)
    if (*p == '"' || *p == '\\' || *p == '{' || *p == '}' || static_cast<unsigned char>(*p) < 0x20) return false;
  return *key != 0;
}

}  // namespace
}  // namespace cb

using namespace cb;

extern "C" {

int cb_tune_key(cb_handle h, char* key, int cap) {
  if (!h || !key || cap <= 0) return fail(h, CB_EINVAL, "bad argument");
  int dev = 0;
  cudaDeviceProp prop;
  CB_CUDA(h, cudaGetDevice(&dev));
  CB_CUDA(h, cudaGetDeviceProperties(&prop, dev));
  unsigned long long* d = nullptr;
  CB_CUDA(h, cudaMallocAsync(&d, sizeof(unsigned long long) * kBits, h->stream));
  unsigned long long hist[kBits] = {};
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long) * kBits, h->stream);
  if (e == cudaSuccess && h->n > 0) {
    const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((h->n + 255) / 256, int64_t(h->num_sms) * 4)));
    k_degree_bits<<<grid, 256, 0, h->stream>>>(h->n, h->rp_id, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) ++h->launches;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hist, d, sizeof hist, cudaMemcpyDeviceToHost, h->stream);
  const cudaError_t ef = cudaFreeAsync(d, h->stream);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "degree histogram");
  unsigned long long total = 0;
  for (unsigned long long v : hist) total += v;
  std::string k = std::string(prop.name) + "|sm" + std::to_string(prop.multiProcessorCount) + "|n" +
                  std::to_string(floor_log2(h->n)) + "|g" + std::to_string(floor_log2(h->nseg)) + "|";
  for (int b = 0; b < kBits; ++b) {
    const long long q = total ? static_cast<long long>((hist[b] * 64.0) / static_cast<double>(total) + 0.5) : 0;
    k += (b ? "," : "") + std::to_string(q);
  }
  for (char& c : k)
    if (c == '"' || c == '\\') c = '_';
  if (static_cast<int>(k.size()) + 1 > cap) return fail(h, CB_ESIZE, "key buffer too small: " + std::to_string(k.size() + 1));
  std::memcpy(key, k.c_str(), k.size() + 1);
  return static_cast<int>(k.size());
}

int cb_tune_cache_lookup(const char* path, const char* key, int64_t* vals, int count) {
  if (!path || !key || !vals || count < 0 || !valid_key(key)) return fail(nullptr, CB_EINVAL, "bad argument");
  std::string text;
  bool exists = false;
  if (!read_file(path, &text, &exists)) return fail(nullptr, CB_EIO, std::string("cannot read ") + path);
  if (exists && !text.empty() && text.find("\"entries\"") == std::string::npos)
    return fail(nullptr, CB_EIO, std::string("not a tuning cache: ") + path);
  size_t b, e;
  find_entry(text, key, &b, &e);
  if (b == std::string::npos) return 0;
  int64_t v[kTuneVals];
  if (!parse_entry(text.substr(b, e - b), v)) return fail(nullptr, CB_EIO, std::string("malformed entry in ") + path);
  const int k = std::min(count, kTuneVals);
  for (int i = 0; i < k; ++i) vals[i] = v[i];
  return k;
}

int cb_tune_cache_store(const char* path, const char* key, const int64_t* vals, int count) {
  if (!path || !key || !vals || count != kTuneVals || !valid_key(key))
    return fail(nullptr, CB_EINVAL, "bad argument");
  std::string text;
  bool exists = false;
  if (!read_file(path, &text, &exists)) return fail(nullptr, CB_EIO, std::string("cannot read ") + path);
  // keep every other well-formed entry; a file that is not this cache's
  // format is left untouched
  std::vector<std::string> entries;
  if (exists && !text.empty()) {
    if (text.find("\"entries\"") == std::string::npos)
      return fail(nullptr, CB_EIO, std::string("not a tuning cache: ") + path);
    size_t at = 0;
    const std::string needle = "\"key\": \"";
    while ((at = text.find(needle, at)) != std::string::npos) {
      const size_t ks = at + needle.size();
      const size_t ke = text.find('"', ks);
      const size_t ob = text.rfind('{', at), oe = text.find('}', at);
      if (ke == std::string::npos || ob == std::string::npos || oe == std::string::npos) break;
      int64_t v[kTuneVals];
      const std::string k = text.substr(ks, ke - ks);
      if (k != key && parse_entry(text.substr(ob, oe + 1 - ob), v)) entries.push_back(format_entry(k, v));
      at = oe + 1;
    }
  }
  entries.push_back(format_entry(key, vals));
  std::string out = "{\"version\": 1, \"entries\": [\n";
  for (size_t i = 0; i < entries.size(); ++i) out += entries[i] + (i + 1 < entries.size() ? ",\n" : "\n");
  out += "]}\n";
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(nullptr, CB_EIO, "cannot write " + tmp);
  const bool ok = std::fwrite(out.data(), 1, out.size(), f) == out.size();
  if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(nullptr, CB_EIO, std::string("cannot write ") + path);
  }
  return CB_OK;
}

int cb_autotune_cached(cb_handle h, uint32_t max_steps, const char* cache_path, int64_t* chosen, int count) {
  if (!h || !cache_path || count < 0) return fail(h, CB_EINVAL, "bad argument");
  char key[512];
  int rc = cb_tune_key(h, key, sizeof key);
  if (rc < 0) return rc;
  int64_t v[kTuneVals];
  rc = cb_tune_cache_lookup(cache_path, key, v, kTuneVals);
  if (rc < 0) return rc;
  int64_t vals[6];
  if (rc == kTuneVals) {
    // settings from the cache: the same checks as cb_set_option
    for (int i = 0; i < kTuneVals; ++i)
      if ((rc = cb_set_option(h, kTuneNames[i], v[i])) != CB_OK) return rc;
    const int64_t got[6] = {v[0], v[1], v[2], v[3], 0, v[4]};
    std::memcpy(vals, got, sizeof got);
  } else {
    rc = cb_autotune(h, max_steps, vals, 6);
    if (rc < 0) return rc;
    const int64_t store[kTuneVals] = {vals[0], vals[1], vals[2], vals[3], vals[5]};
    if ((rc = cb_tune_cache_store(cache_path, key, store, kTuneVals)) != CB_OK) return rc;
  }
  const int k = chosen ? std::min(count, 6) : 0;
  for (int i = 0; i < k; ++i) chosen[i] = vals[i];
  return k;
}

}  // extern "C"
