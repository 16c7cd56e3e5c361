// Spectral propagation (Alg. 6 line 6): E <- sum_{r=0..p} c_r T_r(X) E, the
// Chebyshev series of ProNE's band-pass filter
//   g(L) = exp(-theta/2 [(L - mu I)^2 - I]),   L = I - D^-1 A (Sec. 4.3),
// in the variable X = (L - mu I)^2 / 2 - I (spectrum in [-1, 1] for
// 0 <= mu <= 2): exp(-theta x) = I_0(theta) + 2 sum_{r>=1} (-1)^r I_r(theta)
// T_r(x) with the modified Bessel functions of the first kind I_r, times
// exp(-theta/2).  Defaults p = 10, theta = 0.5, mu = 0.2 (Sec. 5.2).
//
// Every Chebyshev step T_{r+1} = 2 X T_r - T_{r-1} = M (M T_r) - 2 T_r - T_{r-1}
// with M = L - mu I = (1 - mu) I - D^-1 A is two passes of one kernel: a
// warp per row gathers S_i = d_i^-1 sum_j a_ij G_j of the operand G and
// writes  out_i = a G_i + b S_i + c1 W1_i + c2 W2_i,  adding f out_i into the
// running sum F_i, so that no elementwise pass over the n x d matrices is
// needed.  The n x d buffers have a leading dimension of d rounded up to 4;
// their padding columns stay zero.
#include <cmath>
#include <cstring>

#include "sne_internal.cuh"

namespace sne {

namespace {

template <int VPL>
__global__ void __launch_bounds__(256) cheb_spmm_kernel(
    int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ dinv, const float *__restrict__ G,
    int64_t ld, int nvec, float a, float b, const float *W1, float c1, const float *W2, float c2,
    float *out, float *F, float f) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  float4 acc[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t beg = row_ptr[row], end = row_ptr[row + 1];
  for (int64_t p0 = beg; p0 < end; p0 += 32) {
    const int64_t p = p0 + lane;
    int32_t c = 0;
    float w = 0.f;
    if (p < end) {
      c = __ldg(col + p);
      w = val ? __ldg(val + p) : 1.0f;
    }
    const int cnt = (int)min64(32, end - p0);
    int t = 0;
    for (; t + 2 <= cnt; t += 2) {
      const int32_t j0 = __shfl_sync(0xffffffffu, c, t);
      const int32_t j1 = __shfl_sync(0xffffffffu, c, t + 1);
      const float w0 = __shfl_sync(0xffffffffu, w, t);
      const float w1 = __shfl_sync(0xffffffffu, w, t + 1);
      const float4 *r0 = reinterpret_cast<const float4 *>(G + (int64_t)j0 * ld);
      const float4 *r1 = reinterpret_cast<const float4 *>(G + (int64_t)j1 * ld);
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int q = lane + 32 * v;
        if (q < nvec) {
          const float4 x0 = __ldg(r0 + q);
          const float4 x1 = __ldg(r1 + q);
          acc[v].x += w0 * x0.x + w1 * x1.x;
          acc[v].y += w0 * x0.y + w1 * x1.y;
          acc[v].z += w0 * x0.z + w1 * x1.z;
          acc[v].w += w0 * x0.w + w1 * x1.w;
        }
      }
    }
    for (; t < cnt; ++t) {
      const int32_t j0 = __shfl_sync(0xffffffffu, c, t);
      const float w0 = __shfl_sync(0xffffffffu, w, t);
      const float4 *r0 = reinterpret_cast<const float4 *>(G + (int64_t)j0 * ld);
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int q = lane + 32 * v;
        if (q < nvec) {
          const float4 x0 = __ldg(r0 + q);
          acc[v].x += w0 * x0.x;
          acc[v].y += w0 * x0.y;
          acc[v].z += w0 * x0.z;
          acc[v].w += w0 * x0.w;
        }
      }
    }
  }
  const float sb = b * dinv[row];
  const int64_t o = row * ld;
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int q = lane + 32 * v;
    if (q < nvec) {
      const float4 g = *reinterpret_cast<const float4 *>(G + o + 4 * q);
      float4 r = make_float4(a * g.x + sb * acc[v].x, a * g.y + sb * acc[v].y,
                             a * g.z + sb * acc[v].z, a * g.w + sb * acc[v].w);
      if (W1) {
        const float4 x = *reinterpret_cast<const float4 *>(W1 + o + 4 * q);
        r.x += c1 * x.x; r.y += c1 * x.y; r.z += c1 * x.z; r.w += c1 * x.w;
      }
      if (W2) {
        const float4 x = *reinterpret_cast<const float4 *>(W2 + o + 4 * q);
        r.x += c2 * x.x; r.y += c2 * x.y; r.z += c2 * x.z; r.w += c2 * x.w;
      }
      *reinterpret_cast<float4 *>(out + o + 4 * q) = r;
      if (F) {
        float4 *fp = reinterpret_cast<float4 *>(F + o + 4 * q);
        float4 s = *fp;
        s.x += f * r.x; s.y += f * r.y; s.z += f * r.z; s.w += f * r.w;
        *fp = s;
      }
    }
  }
}

// F = c * T (the constant term of the series)
__global__ void scale_copy_kernel(const float *__restrict__ T, float c, int64_t count,
                                  float *__restrict__ F) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride)
    F[q] = c * T[q];
}

cudaError_t launch_cheb_spmm(const sne_csr &g, const float *dinv, const float *G, int64_t ld,
                             int dpad, float a, float b, const float *W1, float c1, const float *W2,
                             float c2, float *out, float *F, float f, cudaStream_t st) {
  const int nvec = dpad / 4;
  const int vpl = (nvec + 31) / 32;
  const unsigned blocks = (unsigned)((g.n + 7) / 8);
  ProfScope ps_(K_PROP, st);
#define SNE_CHEB_CASE(V)                                                                          \
  case V:                                                                                         \
    cheb_spmm_kernel<V><<<blocks, 256, 0, st>>>(g.n, g.row_ptr, g.col_idx, g.val, dinv, G, ld, nvec, \
                                                a, b, W1, c1, W2, c2, out, F, f);                 \
    break;
  switch (vpl) {
    SNE_CHEB_CASE(1)
    SNE_CHEB_CASE(2)
    SNE_CHEB_CASE(3)
    SNE_CHEB_CASE(4)
    SNE_CHEB_CASE(5)
    SNE_CHEB_CASE(6)
    SNE_CHEB_CASE(7)
    SNE_CHEB_CASE(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef SNE_CHEB_CASE
  return cudaGetLastError();
}

}  // namespace

// I_r(theta) = sum_{k>=0} (theta/2)^(2k+r) / (k! (k+r)!), summed until the
// terms fall below the double rounding of the sum.
double bessel_i(int r, double theta) {
  const double h = 0.5 * theta;
  double t = 1.0;
  for (int j = 1; j <= r; ++j) t *= h / j;  // (theta/2)^r / r!
  double s = t;
  for (int k = 1; k < 1000; ++k) {
    t *= h * h / ((double)k * (double)(k + r));
    s += t;
    if (t <= 1e-18 * s) break;
  }
  return s;
}

void propagation_coefficients(int steps, double theta, double *c) {
  const double e = std::exp(-0.5 * theta);
  for (int r = 0; r <= steps; ++r) {
    const double ir = bessel_i(r, theta);
    c[r] = e * (r == 0 ? ir : 2.0 * ((r & 1) ? -ir : ir));
  }
}

size_t propagate_workspace_bytes(int64_t n, int32_t d) {
  const int64_t dpad = (d + 3) / 4 * 4;
  auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return a256(sizeof(Ctrl)) + a256((size_t)n * sizeof(float)) +
         4 * a256((size_t)n * dpad * sizeof(float));
}

int run_propagate(const sne_csr &g, int steps, double theta, double mu, float *E, int64_t lde, int d,
                  void *ws, cudaStream_t st) {
  const int64_t n = g.n;
  const int dpad = (d + 3) / 4 * 4;
  auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char *base = static_cast<char *>(ws);
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(base);
  base += a256(sizeof(Ctrl));
  float *dinv = reinterpret_cast<float *>(base);
  base += a256((size_t)n * sizeof(float));
  const size_t mat = a256((size_t)n * dpad * sizeof(float));
  float *Tprev = reinterpret_cast<float *>(base);
  float *Tcur = reinterpret_cast<float *>(base + mat);
  float *U = reinterpret_cast<float *>(base + 2 * mat);
  float *F = reinterpret_cast<float *>(base + 3 * mat);
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return SNE_ERR_CUDA;
  if (launch_degrees(g, dinv, &ctrl->vol, st) != cudaSuccess) return SNE_ERR_CUDA;
  if (launch_degree_power(dinv, n, -1.0, dinv, 1.0f, st) != cudaSuccess) return SNE_ERR_CUDA;
  // T_0 = E (padding columns zero)
  if (dpad != d && cudaMemsetAsync(Tcur, 0, (size_t)n * dpad * sizeof(float), st) != cudaSuccess)
    return SNE_ERR_CUDA;
  if (cudaMemcpy2DAsync(Tcur, dpad * sizeof(float), E, lde * sizeof(float), d * sizeof(float), n,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SNE_ERR_CUDA;
  double c[1001];
  propagation_coefficients(steps, theta, c);
  const int64_t count = n * dpad;
  {
    ProfScope ps_(K_PROP, st);
    scale_copy_kernel<<<(unsigned)min64(sm_count() * 8, (count + 255) / 256), 256, 0, st>>>(
        Tcur, (float)c[0], count, F);
  }
  if (cudaGetLastError() != cudaSuccess) return SNE_ERR_CUDA;
  const float m1 = (float)(1.0 - mu);
  for (int r = 1; r <= steps; ++r) {
    // U = M T_{r-1}
    if (launch_cheb_spmm(g, dinv, Tcur, dpad, dpad, m1, -1.0f, nullptr, 0.f, nullptr, 0.f, U,
                         nullptr, 0.f, st) != cudaSuccess)
      return SNE_ERR_CUDA;
    cudaError_t e;
    if (r == 1)  // T_1 = X T_0 = M U / 2 - T_0, written over the free buffer
      e = launch_cheb_spmm(g, dinv, U, dpad, dpad, 0.5f * m1, -0.5f, Tcur, -1.0f, nullptr, 0.f,
                           Tprev, F, (float)c[1], st);
    else  // T_r = M U - 2 T_{r-1} - T_{r-2}, written over T_{r-2}
      e = launch_cheb_spmm(g, dinv, U, dpad, dpad, m1, -1.0f, Tcur, -2.0f, Tprev, -1.0f, Tprev, F,
                           (float)c[r], st);
    if (e != cudaSuccess) return SNE_ERR_CUDA;
    std::swap(Tprev, Tcur);
  }
  if (cudaMemcpy2DAsync(E, lde * sizeof(float), F, dpad * sizeof(float), d * sizeof(float), n,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SNE_ERR_CUDA;
  return SNE_OK;
}

}  // namespace sne
