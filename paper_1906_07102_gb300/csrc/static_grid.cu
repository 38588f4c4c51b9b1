// lmg_grid_static: binning plus gridding with all working memory in one fixed-size device
// array of this translation unit, for callers that may not allocate device memory.
//
// The array below is the only device memory this entry point uses besides the caller's
// inputs and output. In host code its name is a host-side stand-in, not a device address,
// so the address is taken with cudaGetSymbolAddress once per device (on the first call
// made with that device current) and carved into the buffers the binning and gridding
// kernels expect. The launches are the same ones lmg_plan_bin and lmg_grid use.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "device_common.cuh"
#include "kernels.h"
#include "lmg_internal.h"

namespace lmg {
namespace {

constexpr int64_t kMaxVis = LMG_STATIC_MAX_VIS;
constexpr int kMaxN = LMG_STATIC_MAX_N;
constexpr int kMaxOversample = LMG_STATIC_MAX_OVERSAMPLE;
constexpr int kRowsPerBlock = 256;
constexpr int kItemTarget = 1024;
constexpr int kStaticStrip = strip_width(LMG_C64);  // complex64 only
constexpr int kMaxStrips = kMaxN / kStaticStrip;
constexpr long long kMaxBuckets = static_cast<long long>(kMaxStrips) * kMaxN;
constexpr int kMaxItems = kMaxStrips * ((kMaxN + kRowsPerBlock - 1) / kRowsPerBlock) +
                          static_cast<int>((2 * kMaxVis) / kItemTarget) + 2;
constexpr int kMaxWp = table_stride(16, LMG_C64);  // float row stride for W <= 16
constexpr int kMaxRing = 18;    // ring slots for W = 16

constexpr size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Byte offsets of the buffers inside the scratch array (sized for the maxima above).
constexpr size_t kOffTable = 0;
constexpr size_t kOffRank = kOffTable + up256(sizeof(float) * (kMaxOversample + 1) * kMaxWp);
constexpr size_t kOffHist = kOffRank + up256(sizeof(int2) * kMaxVis);
constexpr size_t kOffOffsets = kOffHist + up256(sizeof(int) * kMaxBuckets);
constexpr size_t kOffPartial = kOffOffsets + up256(sizeof(int) * (kMaxBuckets + 1));
constexpr size_t kOffRecs = kOffPartial + up256(sizeof(int) * (kMaxBuckets / 4096 + 2));
constexpr size_t kOffItems = kOffRecs + up256(sizeof(Rec) * 2 * kMaxVis);
constexpr size_t kOffCounters = kOffItems + up256(sizeof(Item) * kMaxItems);
constexpr size_t kOffSpill = kOffCounters + up256(sizeof(int) * kNumCounters);
constexpr size_t kScratchBytes = kOffSpill + up256(sizeof(float2) * kMaxItems * kMaxRing * kStaticStrip);

// The working memory: allocated when the library is loaded, on every device that loads
// it, and held until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

struct DeviceSetup {
  bool done = false;
  unsigned char* base = nullptr;  // device address of g_static_scratch
  int sms = 0;
  bool staged = false;            // a table is in the scratch ...
  unsigned long long staged_key = 0;  // ... with this content key (table_key)
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Host staging of the float32 table rows (copied to the scratch when a call brings a table
// that is not the one already staged on its device).
float g_table_host[(kMaxOversample + 1) * kMaxWp];
std::mutex g_table_mutex;

// Content key of a table (FNV-1a over W, oversample, interpolation and the float32 values
// the kernels read): equal keys mean the staged rows can be used as they are.
unsigned long long table_key(const lmg_table* t) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&h](unsigned v) {
    h ^= v;
    h *= 1099511628211ull;
  };
  mix(unsigned(t->W));
  mix(unsigned(t->Ms));
  mix(unsigned(t->interp));
  for (double c : t->C) {
    const float f = float(c);
    unsigned u;
    std::memcpy(&u, &f, sizeof(u));
    mix(u);
  }
  return h;
}

int setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.done) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return set_error(LMG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(LMG_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    s.base = static_cast<unsigned char*>(ptr);
    s.done = true;
  }
  *out = &s;
  return LMG_OK;
}

}  // namespace
}  // namespace lmg

using namespace lmg;

extern "C" int lmg_grid_static(const lmg_table* t, int64_t n_image, double pixel_scale, const double* uv,
                               int64_t nvis, const void* vis, const void* weights, void* grid, void* stream) {
  clear_error();
  if (!t || !grid) return set_error(LMG_EINVAL, "NULL argument");
  if (nvis < 0 || nvis > kMaxVis)
    return set_error(LMG_EINVAL, "nvis must be in [0, " + std::to_string(kMaxVis) + "] for lmg_grid_static");
  if (nvis > 0 && (!uv || !vis)) return set_error(LMG_EINVAL, "uv or vis is NULL");
  if (reinterpret_cast<uintptr_t>(uv) % 16 != 0) return set_error(LMG_EINVAL, "uv must be 16-byte aligned");
  if (!(pixel_scale > 0.0) || !std::isfinite(pixel_scale)) return set_error(LMG_EINVAL, "pixel_scale must be > 0");
  if (t->interp == LMG_INTERP_DIRECT)
    return set_error(LMG_EUNSUPPORTED, "lmg_grid_static runs float32 tables; LMG_INTERP_DIRECT needs a float64 plan");
  if (t->Ms > kMaxOversample)
    return set_error(LMG_EINVAL, "table oversample must be at most " + std::to_string(kMaxOversample) +
                                     " for lmg_grid_static");
  if (n_image < 2 || (n_image & 1)) return set_error(LMG_EINVAL, "n_image must be even and >= 2");
  const double Nd = double(n_image) / t->x0;
  const int64_t N = int64_t(std::llround(Nd));
  if (std::fabs(Nd - double(N)) > 1e-9 * Nd || (N & 1)) return set_error(LMG_EINVAL, "n_image / x0 must be an even integer");
  if (N < 64 || N % kStaticStrip != 0 || N > kMaxN)
    return set_error(LMG_EINVAL, "grid size N = n_image / x0 must be a multiple of 64 in [64, " +
                                     std::to_string(kMaxN) + "] for lmg_grid_static");
  if (N < 2 * t->W) return set_error(LMG_EINVAL, "grid too small for the support width");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(LMG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(LMG_EUNSUPPORTED, "device index out of range");
  DeviceSetup* s = nullptr;
  if (int rc = setup_device(dev, &s)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* base = s->base;
  const int W = t->W, Ms = t->Ms, Wp = table_stride(W, LMG_C64);

  // Table rows in float32, padded to Wp, into the scratch -- only when this device does not
  // already hold this table. The upload copies from pageable host memory, which a stream
  // that is being captured cannot record, so it is refused there.
  {
    std::lock_guard<std::mutex> lock(g_table_mutex);
    const unsigned long long key = table_key(t);
    if (!s->staged || s->staged_key != key) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      e = cudaStreamIsCapturing(st, &cs);
      if (e != cudaSuccess) return set_error(LMG_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
      if (cs != cudaStreamCaptureStatusNone)
        return set_error(LMG_EUNSUPPORTED, "lmg_grid_static would upload a table not yet staged on this device, "
                                           "and the stream is capturing; call it once with this table first");
      for (int i = 0; i <= Ms; ++i)
        for (int j = 0; j < Wp; ++j)
          g_table_host[size_t(i) * Wp + j] = j < W ? float(t->C[size_t(i) * W + j]) : 0.0f;
      e = cudaMemcpyAsync(base + kOffTable, g_table_host, sizeof(float) * size_t(Ms + 1) * Wp, cudaMemcpyHostToDevice,
                          st);
      if (e != cudaSuccess) {
        s->staged = false;
        return set_error(LMG_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));
      }
      s->staged = true;
      s->staged_key = key;
    }
  }

  const int n_strips = int(N / kStaticStrip);
  const int nblk = int((N + kRowsPerBlock - 1) / kRowsPerBlock);
  const int item_cap = n_strips * nblk + int((2 * nvis) / kItemTarget) + 2;
  BinArgs b{};
  b.uv = uv;
  b.nvis = nvis;
  b.scale2 = double(N) * pixel_scale * 4294967296.0;
  b.W = W;
  b.N = int(N);
  b.n_strips = n_strips;
  b.strip = kStaticStrip;
  b.rows_per_block = kRowsPerBlock;
  b.item_target = kItemTarget;
  b.item_cap = item_cap;
  b.max_blocks = s->sms * 8;
  b.rank = reinterpret_cast<int2*>(base + kOffRank);
  b.hist = reinterpret_cast<int*>(base + kOffHist);
  b.offsets = reinterpret_cast<int*>(base + kOffOffsets);
  b.partial = reinterpret_cast<int*>(base + kOffPartial);
  b.recs = reinterpret_cast<Rec*>(base + kOffRecs);
  b.items = reinterpret_cast<Item*>(base + kOffItems);
  b.counters = reinterpret_cast<int*>(base + kOffCounters);
  if (bin_launch(b, st) != 0) return set_error(LMG_ECUDA, std::string("binning launch: ") + cudaGetErrorString(cudaGetLastError()));

  bool tab_smem = false;
  int warps = 8, bps = 0;
  if (sweep_config(W, LMG_C64, Ms, false, 200 * 1024, &tab_smem, &warps))
    return set_error(LMG_EUNSUPPORTED, "sweep shared memory does not fit for this W");
  const size_t smem = sweep_smem_bytes(W, LMG_C64, Ms, tab_smem, false, warps);
  const bool ext = t->interp >= 2;
  if (sweep_set_smem_limits(W, LMG_C64, 0, smem, false, ext) ||
      sweep_occupancy(W, LMG_C64, 0, smem, false, ext, warps, &bps))
    return set_error(LMG_ECUDA, std::string("sweep kernel attributes: ") + cudaGetErrorString(cudaGetLastError()));
  SweepArgs a{};
  a.recs = b.recs;
  a.offsets = b.offsets;
  a.items = b.items;
  a.counters = b.counters;
  a.table = base + kOffTable;
  a.Wp = Wp;
  a.Ms = Ms;
  a.interp = t->interp;
  a.N = int(N);
  a.n_strips = n_strips;
  a.strip = kStaticStrip;
  a.W = W;
  a.dtype = LMG_C64;
  a.accum = 0;
  a.item_cap = item_cap;
  a.grid_blocks = s->sms * (bps > 0 ? bps : 1);
  a.warps = warps;
  a.table_in_smem = tab_smem ? 1 : 0;
  a.vis = vis;
  a.weights = weights;
  a.grid = grid;
  a.spill = base + kOffSpill;
  a.nvis = nvis;
  if (grid_launch(a, st) != 0) return set_error(LMG_ECUDA, std::string("gridding launch: ") + cudaGetErrorString(cudaGetLastError()));
  return LMG_OK;
}
