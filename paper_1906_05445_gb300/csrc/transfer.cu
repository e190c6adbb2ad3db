// transfer.cu -- upload of full FP64 populations into the storage arrays in
// chunks.  The caller's [Q][nodes] array is copied piece by piece into a small
// staging ring on the device and converted there to the stored deviations
// f_i - w_i (scaled for FP16); no device buffer of the whole FP64 field is
// needed, and the copy of one chunk overlaps the conversion of the previous.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

// One chunk: nodes n0 .. n0 + len - 1 of direction i.  Nodes without
// distributions (solid under bounce-back) store 0.
template <typename S, typename T>
__global__ void __launch_bounds__(256) k_upload_chunk(const UploadArgs a, T inv_scale) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.len) return;
  const long long n = a.n0 + k;
  const double v = (a.flags[n] & FL_SOLID) ? 0.0 : a.src[k] - a.w;
  Store<S>::st((S *)a.dst + n, (T)v, inv_scale);
}

long long blocks_of(long long len) { return (len + 255) / 256; }

}  // namespace

void launch_upload_chunk(const UploadArgs &a, int precision, cudaStream_t st) {
  const unsigned g = (unsigned)blocks_of(a.len);
  switch (precision) {
  case LBM_FP64: k_upload_chunk<double, double><<<g, 256, 0, st>>>(a, a.inv_scale); break;
  case LBM_FP32: k_upload_chunk<float, float><<<g, 256, 0, st>>>(a, (float)a.inv_scale); break;
  case LBM_FP32_BF16STORE:
    k_upload_chunk<__nv_bfloat16, float><<<g, 256, 0, st>>>(a, (float)a.inv_scale);
    break;
  default: k_upload_chunk<__half, float><<<g, 256, 0, st>>>(a, (float)a.inv_scale); break;
  }
}

}  // namespace lbm
