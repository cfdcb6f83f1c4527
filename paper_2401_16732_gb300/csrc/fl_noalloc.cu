// fl_he_conv2d_mask_noalloc: the homomorphic convolution + mask of
// fl_he_conv2d_mask for callers that are not allowed to allocate device
// memory -- for example a plugin whose host framework owns every device
// allocation and only hands it input and output buffers, or a real-time
// request loop where an allocation (which can synchronise the whole device)
// must not happen on the request path.
//
// The scratch that fl_he_conv2d_mask takes from the caller (the NTT images
// of the input ciphertexts) lives here in a fixed file-scope device array
// instead.  Every GPU that loads this library holds the array until the
// process exits.  Nothing in this file calls cudaMalloc, cudaFree or any
// other allocating routine.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/flashgpu.h"
#include "fl_launch.h"

namespace {

// Scratch of every call on a device: room for the NTT images of the inputs
// (B * n_in * 2 * L * N 32-bit words).
__device__ __align__(256) static uint32_t g_noalloc_scratch[FL_NOALLOC_SCRATCH_BYTES / 4];

// Host code cannot use &g_noalloc_scratch as a device address (it names a
// host-side shadow).  Resolve the real address with the context's device
// current.  The lookup runs on every call: it is a table lookup once the
// library's device code is loaded, and it stays right after a device reset
// (cudaDeviceReset), which reloads the code at a new address.  On the first
// call on a device it may load that code, so make the first call before any
// stream capture begins.
cudaError_t scratch_for_current_device(uint32_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<uint32_t*>(p);
  return cudaSuccess;
}

}  // namespace

namespace fl {
// Defined in fl_api.cu: the context's parameters and tables, and the
// thread-local error message of fl_last_error().
int ctx_internals(const fl_ctx* ctx, int* logN, int* L, int* device, const uint32_t** tw, const CtxConst** cc);
int fail_msg(int code, const char* fmt, ...);
}  // namespace fl

extern "C" int fl_he_conv2d_mask_noalloc(fl_ctx* ctx, const fl_conv_geom* geom, int B, const uint32_t* w_hat_dev,
                                         const uint32_t* ct_in_dev, const uint32_t* r_dev, uint32_t* ct_out_dev,
                                         void* stream) {
  if (!ctx || !geom) return fl::fail_msg(FL_ERR_ARG, "null context or geometry");
  int logN = 0, L = 0, device = -1;
  const uint32_t* tw = nullptr;
  const fl::CtxConst* cc = nullptr;
  int rc = fl::ctx_internals(ctx, &logN, &L, &device, &tw, &cc);
  if (rc) return rc;
  fl_conv_geom ref;
  if ((rc = fl_conv_geom_make(geom->N, geom->Cin, geom->Cout, geom->H, geom->W, geom->k, geom->stride, geom->pad,
                              &ref)))
    return rc;
  if (memcmp(&ref, geom, sizeof ref) != 0 || geom->N != (1 << logN) || geom->Cout > 65535)
    return fl::fail_msg(FL_ERR_SHAPE, "geometry does not match the context or fl_conv_geom_make");
  if (B < 0) return fl::fail_msg(FL_ERR_ARG, "B=%d", B);
  if (B == 0) return FL_OK;
  const size_t need = fl_he_conv2d_workspace_bytes(ctx, geom, B);
  if (need > FL_NOALLOC_SCRATCH_BYTES)
    return fl::fail_msg(FL_ERR_ARG,
                    "fl_he_conv2d_mask_noalloc: this call needs %zu bytes of scratch, above the fixed %u bytes "
                    "(reduce B or use fl_he_conv2d_mask with a caller-allocated workspace)",
                    need, (unsigned)FL_NOALLOC_SCRATCH_BYTES);
  if (!w_hat_dev || !ct_in_dev || !r_dev || !ct_out_dev) return fl::fail_msg(FL_ERR_ARG, "null device pointer");
  if (((uintptr_t)w_hat_dev | (uintptr_t)ct_in_dev | (uintptr_t)r_dev | (uintptr_t)ct_out_dev) & 15)
    return fl::fail_msg(FL_ERR_ARG, "device pointers must be 16-byte aligned");
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess || cur != device) return fl::fail_msg(FL_ERR_ARG, "current device is not the context's device");
  uint32_t* scratch = nullptr;
  if ((e = scratch_for_current_device(&scratch)) != cudaSuccess)
    return fl::fail_msg(FL_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
  // The forward NTT writes every scratch word the contraction later reads,
  // so nothing left by an earlier call needs clearing.
  cudaStream_t st = (cudaStream_t)stream;
  const int rows = B * geom->n_in * 2 * L;
  if ((e = fl::launch_ntt_fwd(logN, rows, ct_in_dev, rows, 0, scratch, rows, 0, 1, tw, *cc, st)) != cudaSuccess)
    return fl::fail_msg(FL_ERR_CUDA, "input ntt: %s", cudaGetErrorString(e));
  fl::ConvDims cd{geom->Cout, geom->G, geom->n_in, geom->n_out, geom->bands};
  if ((e = fl::launch_conv_intt(logN, B, cd, w_hat_dev, scratch, ct_out_dev, r_dev, tw, *cc, st, true)) !=
      cudaSuccess)
    return fl::fail_msg(FL_ERR_CUDA, "contraction + intt: %s", cudaGetErrorString(e));
  return FL_OK;
}
