// xy_static.cu -- cluster labeling of caller-supplied bonds that allocates
// nothing: its scratch lives in a fixed array compiled into the library.
//
// Who this is for: callers that cannot allocate device memory, and so cannot
// hand xy_init the workspace a lattice handle needs -- for example a plugin
// that its host application gives only the input and output buffers, or a
// real-time loop whose rules forbid device allocation once it runs.  They
// pass device pointers to the bonds and to the output labels; everything
// else comes from `g_label_scratch` below.
//
// The scratch array is a file-scope __device__ array, so every GPU that
// loads this library holds it (about 1.05 MB) until the process exits.  All
// calls share it and it keeps the contents of the last call: every call
// rewrites the parts it reads (descriptor, state word, bit planes, tile edge
// table, link list) before using them, and calls whose work overlaps on the GPU (two streams, or two
// host threads at once) race on it and give wrong labels.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/xy.h"
#include "layout.cuh"
#include "sweep_kernels.cuh"

using namespace xyk;

namespace {

constexpr uint32_t kStaticTile = 32;  // labeling tile 32 x 32
constexpr uint32_t kStaticMaxTiles =
    (XY_STATIC_MAX_L / 32) * (XY_STATIC_MAX_L / kStaticTile);
constexpr size_t kPlaneWords = static_cast<size_t>(kStaticMaxTiles) * kStaticTile;

// layout of the scratch array (byte offsets, each 256-aligned)
constexpr size_t kOffDesc = 0;
constexpr size_t kOffPrefix = 256;
constexpr size_t kOffState = 512;
constexpr size_t kOffRplane = 1024;
constexpr size_t kOffDplane = kOffRplane + kPlaneWords * sizeof(uint32_t);
constexpr size_t kOffEdge = kOffDplane + kPlaneWords * sizeof(uint32_t);
constexpr size_t kOffLinks =
    kOffEdge + static_cast<size_t>(kStaticMaxTiles) * edge_words<kStaticTile>() * sizeof(uint32_t);
constexpr size_t kOffLinkCount =
    kOffLinks + static_cast<size_t>(kStaticMaxTiles) * (kStaticTile + 32) * sizeof(uint32_t);
constexpr size_t kScratchBytes = kOffLinkCount + static_cast<size_t>(kStaticMaxTiles) * sizeof(uint32_t);
static_assert(sizeof(LatDesc) <= 256 && sizeof(DevState) <= 512, "scratch layout");

// The scratch memory.  In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_label_scratch[kScratchBytes];

xy_status fail(xy_status s, const char *fmt, ...) {
  char msg[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  xy_set_last_error_message(msg);  // read back through xy_last_error()
  return s;
}

// Device address of the scratch on each device.  It is looked up (with that
// device current) by the first call on the device, and looked up again by
// every call made outside stream capture: a cudaDeviceReset ends the context
// the address belonged to, and the next call outside capture then picks up
// the address in the new context.  A call made while its stream is being
// captured uses the address of the last call outside capture.
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

xy_status scratch_for_current_device(cudaStream_t stream, unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(XY_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(XY_EUNSUPPORTED, "device %d out of range", dev);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return fail(XY_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev] || cap == cudaStreamCaptureStatusNone) {
    if (cap != cudaStreamCaptureStatusNone)
      return fail(XY_EINVAL, "the first call on a device must come before any stream capture");
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_label_scratch);
    if (e != cudaSuccess)
      return fail(XY_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_ptr[dev];
  return XY_OK;
}

// Write the descriptor, the work prefix and a zeroed state word into the
// scratch (values travel as kernel arguments, so no host buffer must outlive
// the call).
__global__ void k_static_setup(LatDesc d, LatDesc *d_desc, uint32_t *d_prefix) {
  *d_desc = d;
  d_prefix[0] = 0u;
  d_prefix[1] = d.ntiles;
  *d.st = DevState{};  // error word (and everything else) starts at zero
}

// Pack byte bonds into the tile-major bit planes: one warp per tile row.
__global__ void k_static_pack(const uint8_t *__restrict__ right,
                              const uint8_t *__restrict__ down, LatDesc d) {
  const uint64_t gw = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const uint64_t rows = static_cast<uint64_t>(d.ntiles) * kStaticTile;
  if (gw >= rows) return;
  const uint32_t tile = static_cast<uint32_t>(gw / kStaticTile);
  const uint32_t r = static_cast<uint32_t>(gw % kStaticTile);
  const Tile g = tile_geom<kStaticTile>(d.L, d.ntx, d.ntx_magic, tile);
  bool br = false, bd = false;
  if (r < g.h && lane < static_cast<int>(g.w)) {
    const uint64_t i = static_cast<uint64_t>(g.y0 + r) * d.L + g.x0 + lane;
    br = right[i] != 0;
    bd = down[i] != 0;
  }
  const uint32_t R = __ballot_sync(0xFFFFFFFFu, br);
  const uint32_t D = __ballot_sync(0xFFFFFFFFu, bd);
  if (lane == 0) {
    d.rplane[gw] = R;
    d.dplane[gw] = D;
  }
}

}  // namespace

extern "C" {

xy_status xy_label_bonds_static(uint32_t L, const uint8_t *d_right, const uint8_t *d_down,
                                uint32_t *d_labels, void *cuda_stream, int sync) {
  if (L < 2 || L > XY_STATIC_MAX_L)
    return fail(XY_EINVAL, "L = %u outside 2..%u (the size of the built-in scratch)", L,
                XY_STATIC_MAX_L);
  if (!d_right || !d_down || !d_labels) return fail(XY_EINVAL, "NULL device pointer");
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  unsigned char *scratch = nullptr;
  xy_status s = scratch_for_current_device(stream, &scratch);
  if (s != XY_OK) return s;

  LatDesc d{};
  d.L = L;
  d.Lmagic = ~0ull / L + 1ull;
  d.inv_n = 1.0 / (static_cast<double>(L) * L);
  d.ntx = (L + 31) / 32;
  d.ntx_magic = ~0ull / d.ntx + 1ull;
  d.nty = (L + kStaticTile - 1) / kStaticTile;
  d.ntiles = d.ntx * d.nty;
  d.label = d_labels;
  d.rplane = reinterpret_cast<uint32_t *>(scratch + kOffRplane);
  d.dplane = reinterpret_cast<uint32_t *>(scratch + kOffDplane);
  d.edge = reinterpret_cast<uint32_t *>(scratch + kOffEdge);
  d.links = reinterpret_cast<uint32_t *>(scratch + kOffLinks);
  d.link_count = reinterpret_cast<uint32_t *>(scratch + kOffLinkCount);
  d.st = reinterpret_cast<DevState *>(scratch + kOffState);
  d.find_cap = kFindCap;
  d.link_cap = kStaticTile + 32u;
  LatDesc *d_desc = reinterpret_cast<LatDesc *>(scratch + kOffDesc);
  uint32_t *d_prefix = reinterpret_cast<uint32_t *>(scratch + kOffPrefix);
  const uint32_t nw = d.ntiles;

  k_static_setup<<<1, 1, 0, stream>>>(d, d_desc, d_prefix);
  const uint64_t rows = static_cast<uint64_t>(nw) * kStaticTile;
  k_static_pack<<<static_cast<uint32_t>((rows * 32 + 255) / 256), 256, 0, stream>>>(d_right,
                                                                                  d_down, d);
  k_bond_label<kStaticTile, float, true, true>
      <<<nw, kThreads, bond_label_smem<kStaticTile>(), stream>>>(d_desc, d_prefix, 1, nw, 0u, LatDesc{});
  const uint64_t items = static_cast<uint64_t>(nw) * (kStaticTile + 32);
  const uint32_t eb = static_cast<uint32_t>((items + kThreads - 1) / kThreads);
  k_merge<kStaticTile><<<eb, kThreads, 0, stream>>>(d_desc, d_prefix, 1, nw, LatDesc{});
  k_compress<kStaticTile>
      <<<compress_blocks(nw), kThreads, 0, stream>>>(d_desc, d_prefix, 1, nw, LatDesc{});
  k_flip_measure<kStaticTile, float, true>
      <<<nw, kThreads, flip_smem<kStaticTile>(), stream>>>(d_desc, d_prefix, 1, nw, 0u, LatDesc{});
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(XY_ECUDA, "launch: %s", cudaGetErrorString(e));
  if (!sync) return XY_OK;
  e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail(XY_ECUDA, "synchronize: %s", cudaGetErrorString(e));
  uint32_t err = 0;
  e = cudaMemcpy(&err, &d.st->err, sizeof(err), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(XY_ECUDA, "error word: %s", cudaGetErrorString(e));
  return device_error_status(err);  // the setup kernel clears the word on every call
}

}  // extern "C"
