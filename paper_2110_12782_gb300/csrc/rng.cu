// Random draws of the method: the Gaussian test matrix of Alg. 5 and the
// sparse-sign matrices of Alg. 3, plus the unique() of Alg. 3 line 8.
#include <climits>

#include "sne_internal.cuh"

namespace sne {

// Omega = randn(n, cols) (Alg. 5 line 3).  Entry e = i*cols + c is taken from
// the pair of draws 2*(e/2), 2*(e/2)+1 by Box-Muller on 24-bit uniforms:
// u1 = (x1>>40 + 1) 2^-24 in (0, 1], u2 = (x2>>40) 2^-24, r = sqrt(-2 ln u1),
// even e -> r cos(2 pi u2), odd e -> r sin(2 pi u2).
__global__ void gaussian_kernel(int64_t n, int32_t cols, uint64_t key, float *__restrict__ out,
                                int64_t ld) {
  const int64_t total = n * (int64_t)cols;
  const int64_t npairs = (total + 1) >> 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t pr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pr < npairs; pr += stride) {
    const uint64_t x1 = draw(key, 2 * (uint64_t)pr);
    const uint64_t x2 = draw(key, 2 * (uint64_t)pr + 1);
    const float u1 = (float)((x1 >> 40) + 1) * 0x1p-24f;
    const float u2 = (float)(x2 >> 40) * 0x1p-24f;
    const float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    const int64_t e0 = 2 * pr;
    int64_t i = e0 / cols, c = e0 - i * cols;
    out[i * ld + c] = r * cs;
    if (e0 + 1 < total) {
      if (++c == cols) {
        c = 0;
        ++i;
      }
      out[i * ld + c] = r * sn;
    }
  }
}

cudaError_t launch_gaussian(int64_t n, int32_t cols, uint64_t seed, int32_t stream_id, float *out,
                            int64_t ld, cudaStream_t st) {
  const int64_t npairs = (n * (int64_t)cols + 1) / 2;
  if (npairs <= 0) return cudaSuccess;
  int64_t blocks = (npairs + 255) / 256;
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  ProfScope ps_(K_RNG, st);
  gaussian_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, cols, stream_key(seed, stream_id), out, ld);
  return cudaGetLastError();
}

// Alg. 3 lines 4-6, one thread per column j.  Rows: Lemire's multiply-shift
// with rejection on draws (j << 32) + c, c = 0, 1, ..., skipping rows already
// taken in the column (randperm(n, z)); sign t: top bit of draw((j<<32)|(1<<31)|t).
constexpr int kMaxZ = 64;
__global__ void sparse_sign_kernel(int64_t n, int32_t cols, int32_t z, uint64_t key,
                                   int32_t *__restrict__ idx, int8_t *__restrict__ sign,
                                   Ctrl *ctrl) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  const uint64_t un = (uint64_t)n;
  const uint64_t base = (uint64_t)j << 32;
  uint64_t ctr = base;
  const uint64_t threshold = (0ull - un) % un;  // (2^64 - n) mod n
  int32_t chosen[kMaxZ];
  for (int t = 0; t < z; ++t) {
    for (;;) {
      uint64_t x = draw(key, ctr++);
      uint64_t lo = x * un;
      uint64_t hi = __umul64hi(x, un);
      if (lo < un) {
        while (lo < threshold) {
          x = draw(key, ctr++);
          lo = x * un;
          hi = __umul64hi(x, un);
        }
      }
      const int32_t r = (int32_t)hi;
      bool dup = false;
      for (int s = 0; s < t; ++s) dup |= (chosen[s] == r);
      if (!dup) {
        chosen[t] = r;
        break;
      }
      if (ctr - base > (1ull << 30)) {  // cannot happen for z <= n; bounded anyway
        record_error(ctrl, SNE_ERR_NUMERIC, W_SPARSE_SIGN);
        chosen[t] = r;
        break;
      }
    }
  }
  for (int t = 0; t < z; ++t) {
    idx[(int64_t)j * z + t] = chosen[t];
    const uint64_t bit = draw(key, base | (1ull << 31) | (uint64_t)t) >> 63;
    sign[(int64_t)j * z + t] = bit ? (int8_t)-1 : (int8_t)1;
  }
}

cudaError_t launch_sparse_sign(int64_t n, int32_t cols, int32_t z, uint64_t seed, int32_t stream_id,
                               int32_t *idx, int8_t *sign, Ctrl *ctrl, cudaStream_t st) {
  if (cols <= 0) return cudaSuccess;
  ProfScope ps_(K_RNG, st);
  sparse_sign_kernel<<<(cols + 127) / 128, 128, 0, st>>>(n, cols, z, stream_key(seed, stream_id),
                                                         idx, sign, ctrl);
  return cudaGetLastError();
}

// unique(): one CTA sorts the keys (bitonic sort in shared memory), keeps the
// first of every run, and maps every input key to its position in the result.
__global__ void __launch_bounds__(1024) unique_kernel(const int32_t *__restrict__ keys, int32_t count,
                                                      int32_t P, int32_t *__restrict__ uniq,
                                                      int32_t *__restrict__ nuniq,
                                                      int32_t *__restrict__ pos) {
  extern __shared__ int32_t s[];  // P keys + 1024 + 32 scan slots
  int32_t *scan = s + P;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < P; i += nt) s[i] = i < count ? keys[i] : INT_MAX;
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < P / 2; i += nt) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const int32_t a = s[lo], b = s[hi];
        if ((a > b) == up) {
          s[lo] = b;
          s[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  // each thread owns a contiguous segment of the sorted array
  const int seg = (P + nt - 1) / nt;
  const int b0 = tid * seg, b1 = min(P, b0 + seg);
  int cnt = 0;
  for (int i = b0; i < b1; ++i)
    cnt += (s[i] != INT_MAX && (i == 0 || s[i] != s[i - 1])) ? 1 : 0;
  // block exclusive scan of cnt
  const int lane = tid & 31, warp = tid >> 5;
  int v = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) scan[1024 + warp] = v;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (nt >> 5) ? scan[1024 + lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    scan[1024 + lane] = w;  // inclusive over warps
  }
  __syncthreads();
  int off = v - cnt + (warp > 0 ? scan[1024 + warp - 1] : 0);
  for (int i = b0; i < b1; ++i)
    if (s[i] != INT_MAX && (i == 0 || s[i] != s[i - 1])) uniq[off++] = s[i];
  if (tid == nt - 1) *nuniq = off;
  __syncthreads();
  __threadfence_block();
  const int total = scan[1024 + (nt >> 5) - 1];
  // positions by binary search in the unique array
  for (int i = tid; i < count; i += nt) {
    const int32_t key = keys[i];
    int lo = 0, hi = total - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (uniq[mid] < key) lo = mid + 1;
      else hi = mid;
    }
    pos[i] = lo;
  }
}

cudaError_t launch_unique(const int32_t *keys, int32_t count, int32_t *uniq, int32_t *nuniq,
                          int32_t *pos, Ctrl *ctrl, int32_t where, cudaStream_t st) {
  (void)ctrl;
  (void)where;
  if (count <= 0 || count > kUniqueMax) return cudaErrorInvalidValue;
  int P = 2;
  while (P < count) P <<= 1;
  const size_t smem = (size_t)(P + 1024 + 32) * sizeof(int32_t);
  cudaError_t e = cudaFuncSetAttribute(unique_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  ProfScope ps_(K_UNIQUE, st);
  unique_kernel<<<1, 1024, smem, st>>>(keys, count, P, uniq, nuniq, pos);
  return cudaGetLastError();
}

}  // namespace sne
