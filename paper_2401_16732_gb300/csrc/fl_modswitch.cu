// BFV modulus switching on the GPU: drop the last RNS primes of a ciphertext
// with rounding (Fan and Vercauteren's scale-and-round by q'/q), one prime at
// a time.  For the dropped prime p and each kept prime q_i:
//   y   = [x]_p as a centred integer in (-p/2, p/2]
//   x_i <- (x_i - y) * p^-1 mod q_i
// (x - y) / p is then exactly the nearest integer to x / p (p is odd, so
// there is no tie).  It serves only to shrink output ciphertexts before they
// leave the device: the paper keeps one modulus throughout.
#include <cuda_runtime.h>

#include "fl_device.cuh"
#include "fl_launch.h"

namespace fl {

// One thread per coefficient of one component: its L residues are N words
// apart, so a warp reads and writes 128 contiguous bytes per limb.
__global__ void k_mod_switch(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, long long rows, int N,
                             ModSwitchConst mc) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)rows * N) return;
  const size_t row = idx / N, u = idx % N;
  const int L = mc.L, Lo = mc.L_out;
  uint32_t x[FL_MAX_L];
#pragma unroll
  for (int l = 0; l < FL_MAX_L; ++l) x[l] = l < L ? __ldcs(in + (row * L + l) * N + u) : 0;
#pragma unroll
  for (int d = FL_MAX_L - 1; d >= 1; --d) {
    if (d >= L || d < Lo) continue;
    const uint32_t p = mc.q[d], y = x[d];
    const bool neg = y > (p >> 1);
    const uint32_t a = neg ? p - y : y;  // |centred y| <= p/2 < q_i
#pragma unroll
    for (int i = 0; i < FL_MAX_L - 1; ++i) {
      if (i >= d) continue;
      const uint32_t qi = mc.q[i];
      const uint32_t t = neg ? x[i] + a : x[i] + qi - a;  // x_i - y mod q_i, in [0, 2 q_i)
      x[i] = csub(shoup_mul(t, mc.inv[d][i], mc.inv_sh[d][i], qi), qi);
    }
  }
#pragma unroll
  for (int l = 0; l < FL_MAX_L; ++l)
    if (l < Lo) __stcs(out + (row * Lo + l) * N + u, x[l]);
}

cudaError_t launch_mod_switch(const uint32_t* in, uint32_t* out, long long rows, int N, const ModSwitchConst& mc,
                              cudaStream_t st) {
  const size_t total = (size_t)rows * N;
  if (total == 0) return cudaSuccess;
  k_mod_switch<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(in, out, rows, N, mc);
  return cudaGetLastError();
}

}  // namespace fl
