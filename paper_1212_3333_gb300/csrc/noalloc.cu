// amr_render_host_noalloc: a host-buffer render that allocates no device memory.
//
// Some callers cannot call cudaMalloc on the render path: a renderer embedded in a host
// application whose device memory is owned and capped by another allocator, a process
// that must not grow its device footprint after start-up, or code that is not allowed to
// synchronise the device the way cudaMalloc/cudaFree may.  amr_render_host stages the
// transfer function and the image in device buffers it allocates on first use; this entry
// point stages them in one fixed array that is part of the library image instead.
//
// The array (kScratchBytes = 4 MiB + 32 KiB + 64 B) is a file-scope __device__ variable,
// so every GPU that loads the library holds it until the process exits.  Layout:
//   [0, 64)          kernel counters (samples, status, exact-path counts), zeroed per call
//   [64, 64 + 32K)   transfer function, up to 2048 RGBA entries
//   [.., + 4 MiB)    image band: rows of the frame rendered per launch
// The frame is rendered in bands of whole 16-row tiles that fit the band buffer and each
// band is copied to the caller's host image, so the image size is not limited; one row must
// fit (width <= 16384 pixels).  Calls that overlap on the GPU (several streams or threads at
// once) share the array and race; serialise them.
//
// With CUDA's lazy module loading the array is committed when this file's module is first
// used on a device, i.e. by the first call there (the address lookup); a caller whose
// footprint must be fixed before rendering makes one call at start-up.  The looked-up
// address is cached per device ordinal; cudaDeviceReset invalidates it, as it does every
// context's device memory (such contexts must be destroyed, not rendered).
#include <cstring>
#include <mutex>

#include "ctx.h"

namespace amr {
namespace {

constexpr size_t kCounterBytes = kNumCounters * sizeof(unsigned long long);
constexpr size_t kTfMax = 2048;
constexpr size_t kTfBytes = kTfMax * sizeof(float4);
constexpr size_t kBandBytes = (size_t)4 << 20;
constexpr size_t kScratchBytes = kCounterBytes + kTfBytes + kBandBytes;
constexpr int kTileRows = 16;  // rows of one block tile: bands stay tile-aligned

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_setup_mutex;
constexpr int kMaxDevices = 256;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (the host-side symbol is only a
// stand-in, never a device address).  Looked up once per device.  The current device must
// be the one the context was uploaded to: the kernel reads the context's tree and bricks
// there, so scratch on another device would be a foreign address.
amr_status scratch_address(amr_ctx* c, void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(c, AMR_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(c, AMR_ERR_CUDA, "device ordinal out of range");
  if (dev != c->dev.device)
    return fail(c, AMR_ERR_STATE, "the current device is not the one the context was built on");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return fail(c, AMR_ERR_CUDA,
                  std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return AMR_OK;
}

}  // namespace
}  // namespace amr

using namespace amr;

extern "C" amr_status amr_render_host_noalloc(amr_ctx* c, const amr_camera* cam,
                                              const float* tf_rgba_host, int32_t tf_n,
                                              const amr_render_params* params_in,
                                              float* out_rgba_host, void* cuda_stream,
                                              uint64_t* samples_out) {
  if (!c) return AMR_ERR_ARG;
  if (!c->device_built) return fail(c, AMR_ERR_STATE, "render before amr_build_kdtree");
  if (!cam || !params_in || !tf_rgba_host || !out_rgba_host)
    return fail(c, AMR_ERR_ARG, "NULL argument");
  // the schedule follows the whole frame, not the bands it is rendered in
  const amr_render_params resolved = resolve_render_schedule(cam, *params_in);
  const amr_render_params* params = &resolved;
  if (tf_n < 2 || (size_t)tf_n > kTfMax)
    return fail(c, AMR_ERR_ARG, "tf_n must be in [2, 2048] (the no-alloc staging limit)");
  if (cam->width <= 0 || (size_t)cam->width * sizeof(float4) * kTileRows > kBandBytes)
    return fail(c, AMR_ERR_ARG,
                "image width must be in [1, 16384] (one 16-row band must fit the 4 MiB staging)");
  if (params->row0 < 0 || params->row0 >= cam->height)
    return fail(c, AMR_ERR_ARG, "row0 out of range");
  void* base = nullptr;
  amr_status s = scratch_address(c, &base);
  if (s != AMR_OK) return s;
  unsigned long long* counters = reinterpret_cast<unsigned long long*>(base);
  float4* tf_dev = reinterpret_cast<float4*>(static_cast<char*>(base) + kCounterBytes);
  float4* band = reinterpret_cast<float4*>(static_cast<char*>(base) + kCounterBytes + kTfBytes);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int first = params->row0;
  const int total =
      params->rows <= 0 ? cam->height - first : std::min(params->rows, cam->height - first);
  const int band_rows =
      (int)(kBandBytes / ((size_t)cam->width * sizeof(float4)) / kTileRows) * kTileRows;
  // once work is queued, an error return first waits for it: the queued copies write the
  // caller's host image, which the caller may free as soon as the call returns
  auto drain = [&](amr_status r) {
    cudaStreamSynchronize(st);
    return r;
  };
#define CKN(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return drain(fail(c, AMR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); \
  } while (0)
  // the array keeps the previous call's contents: start the counters from zero
  CKN(cudaMemsetAsync(counters, 0, kCounterBytes, st));
  CKN(cudaMemcpyAsync(tf_dev, tf_rgba_host, (size_t)tf_n * sizeof(float4), cudaMemcpyHostToDevice,
                      st));
  for (int r = 0; r < total; r += band_rows) {
    amr_render_params p = *params;
    p.row0 = first + r;
    p.rows = std::min(band_rows, total - r);
    RenderArgs a;
    s = prepare_render_args(c, cam, tf_n, &p, &a);
    if (s != AMR_OK) return drain(s);
    a.tf = tf_dev;
    a.out = band;
    a.counters = counters;
    a.ray.counters = counters;
    s = launch_render_args(c, a, &p, cuda_stream);
    if (s != AMR_OK) return drain(s);
    CKN(cudaMemcpyAsync(out_rgba_host + (size_t)r * cam->width * 4, band,
                        (size_t)p.rows * cam->width * sizeof(float4), cudaMemcpyDeviceToHost, st));
  }
  unsigned long long h[kNumCounters] = {0};
  CKN(cudaMemcpyAsync(h, counters, sizeof h, cudaMemcpyDeviceToHost, st));
  CKN(cudaStreamSynchronize(st));
#undef CKN
  if (samples_out) *samples_out = h[0];
  if (h[1] & kStatusDevice) return fail(c, AMR_ERR_DEVICE, "device reported a malformed tree");
  if (h[1] & kStatusCapacity)
    return fail(c, AMR_ERR_CAPACITY, "a ray exceeded the segment or sample bound");
  return AMR_OK;
}
