// ac_noalloc.cu -- colour means without any device allocation.
//
// Some callers cannot call cudaMalloc: real-time or embedded pipelines that
// forbid device allocation once they are running, and code that lives under a
// framework's fixed device-memory budget (a caching allocator that owns all
// free memory).  ac_colour_means_static serves them: it computes the colour
// means c_i = int u_i I / int u_i straight from the phase field and the image,
// and keeps the block partials of its FP64 reduction in a file-scope
// __device__ array instead of in allocated scratch.
//
// The array is g_means_scratch below: kStaticBlocks rows of 4*AC_MAX_PHASES
// partial sums plus one row of totals, 132 KiB.  Every GPU that loads this
// library holds it until the process exits.  In host code its name is only a
// host-side stand-in, never a device address, so the address is looked up
// once per device with cudaGetSymbolAddress (see scratch_for_current_device).
#include <mutex>
#include <string>

#include "../../include/ac.h"
#include "ac_kernels.cuh"

namespace ac {
void set_last_error(const char *msg);  // ac_api.cu: the message ac_last_error() returns
}

namespace {

constexpr int kStaticBlocks = 512;
constexpr int kStaticCols = 4 * AC_MAX_PHASES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_means_scratch[(kStaticBlocks + 1) * kStaticCols];

int noalloc_fail(int code, const std::string &msg) {
  ac::set_last_error(msg.c_str());
  return code;
}

// Per-node image moments gathered from the (up to) four pixels around the
// node, as in k_moments: m1 = (2 I(x,y) + 2 I(x-1,y-1) + I(x-1,y) + I(x,y-1))/6.
template <int N>
__global__ void __launch_bounds__(ac::kBlock) k_means_image_partial(const double *__restrict__ u,
                                                                    const float *__restrict__ img, ac::Geo g,
                                                                    double *__restrict__ part) {
  double acc[4 * N];
#pragma unroll
  for (int k = 0; k < 4 * N; ++k) acc[k] = 0.0;
  const int64_t n = (int64_t)g.Wn * (g.H + 1);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(k % g.Wn), y = (int)(k / g.Wn);
    const double m0 = g.m0[ac::node_class(g, x, y)];
    double s[3] = {0, 0, 0};
    const int px[4] = {x, x - 1, x, x - 1};
    const int py[4] = {y, y - 1, y - 1, y};
    const double w[4] = {2.0, 2.0, 1.0, 1.0};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (px[q] < 0 || px[q] >= g.W || py[q] < 0 || py[q] >= g.H) continue;
      const float *p = img + ((int64_t)py[q] * g.W + px[q]) * 3;
      s[0] += w[q] * (double)p[0];
      s[1] += w[q] * (double)p[1];
      s[2] += w[q] * (double)p[2];
    }
    double uk[N];
    ac::ldn<double, N>(u + k * N, uk);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      acc[0 * N + i] += uk[i] * m0;
      acc[1 * N + i] += uk[i] * (s[0] / 6.0);
      acc[2 * N + i] += uk[i] * (s[1] / 6.0);
      acc[3 * N + i] += uk[i] * (s[2] / 6.0);
    }
  }
  ac::block_sum_store<4 * N>(acc, part + (int64_t)blockIdx.x * 4 * N);
}

// c_i = s_i / mass_i; a phase of zero mass gets c_i = 0.
template <int N>
__global__ void k_means_static_finish(const double *__restrict__ tot, double *__restrict__ c) {
  const int i = threadIdx.x;
  if (i >= N) return;
  const double mass = tot[i];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) c[i * 3 + ch] = mass != 0.0 ? tot[(1 + ch) * N + i] / mass : 0.0;
}

template <int N>
void launch(const double *u, const float *img, const ac::Geo &g, double *scratch, double *c, cudaStream_t s) {
  const int64_t n = (int64_t)g.Wn * (g.H + 1);
  const int64_t b = (n + ac::kBlock - 1) / ac::kBlock;
  const int blocks = (int)(b < kStaticBlocks ? b : kStaticBlocks);
  double *part = scratch, *tot = scratch + (int64_t)kStaticBlocks * kStaticCols;
  k_means_image_partial<N><<<blocks, ac::kBlock, 0, s>>>(u, img, g, part);
  ac::k_colsum<<<4 * N, ac::kBlock, 0, s>>>(part, blocks, 4 * N, tot);
  k_means_static_finish<N><<<1, 32, 0, s>>>(tot, c);
}

// The device address of g_means_scratch on the current device, looked up
// with cudaGetSymbolAddress the first time a device is seen (with that device
// current) and cached per device.
int scratch_for_current_device(double **out) {
  static std::mutex mu;
  static double *addr[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(AC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(AC_ERR_ARG, "device ordinal beyond the supported 64 devices");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_means_scratch);
    if (e != cudaSuccess)
      return noalloc_fail(AC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    addr[dev] = static_cast<double *>(p);
  }
  *out = addr[dev];
  return AC_OK;
}

}  // namespace

extern "C" int ac_colour_means_static(const double *u, const float *rgb, int width, int height, int n_phases,
                                      double *c, void *stream) {
  if (!u || !rgb || !c) return noalloc_fail(AC_ERR_ARG, "NULL argument");
  if (width < 1 || height < 1 || (int64_t)(width + 1) * (height + 1) > (int64_t)1 << 31)
    return noalloc_fail(AC_ERR_ARG, "image size must be >= 1x1 with at most 2^31 nodes");
  if (n_phases < 2 || n_phases > AC_MAX_PHASES)
    return noalloc_fail(AC_ERR_ARG, "n_phases must be in [2, 8]: the static scratch holds 4*8 sums per block");
  double *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  ac::Geo g{};
  g.W = width;
  g.H = height;
  g.Wn = width + 1;
  const int xs[3] = {0, 1, width}, ys[3] = {0, 1, height};
  for (int cy = 0; cy < 3; ++cy)
    for (int cx = 0; cx < 3; ++cx) {
      const int x = xs[cx], y = ys[cy];
      auto pix = [&](int px, int py) { return (int)(px >= 0 && px < width && py >= 0 && py < height); };
      g.m0[cy * 3 + cx] = (2 * pix(x, y) + pix(x - 1, y) + pix(x, y - 1) + 2 * pix(x - 1, y - 1)) / 6.0;
    }
  cudaStream_t s = (cudaStream_t)stream;
  switch (n_phases) {
    case 2: launch<2>(u, rgb, g, scratch, c, s); break;
    case 3: launch<3>(u, rgb, g, scratch, c, s); break;
    case 4: launch<4>(u, rgb, g, scratch, c, s); break;
    case 5: launch<5>(u, rgb, g, scratch, c, s); break;
    case 6: launch<6>(u, rgb, g, scratch, c, s); break;
    case 7: launch<7>(u, rgb, g, scratch, c, s); break;
    default: launch<8>(u, rgb, g, scratch, c, s); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(AC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return AC_OK;
}
