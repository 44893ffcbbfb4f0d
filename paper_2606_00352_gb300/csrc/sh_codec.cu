// 32-byte packed SH representation (Sec. 4.2): encoding at scene creation.
//   transform  YCoCg-R lifting per basis: Co = R - B, t = B + Co/2,
//              Cg = G - t, Y = t + Cg/2
//   scales     per basis and channel, the 99.5th percentile of |value| over
//              the scene's gaussians (histogram of 4096 bins below the
//              channel's maximum; the upper edge of the bin holding it)
//   quantise   bases 1..15: x = clamp(v / s, -1, 1), g = sign(x) sqrt(|x|),
//              q = rint(g Q), Q = 2^(bits-1) - 1 (Y 6, Co 4, Cg 4 bits);
//              basis 0: Y as float16 bits, Co and Cg linear:
//              q = rint(clamp(v / s, -1, 1) 4095) in 13 bits
//   layout     fields in order from bit 0 of word 0 (8 uint32 words)
// Decoding runs in the projection (sh_codec.cuh).
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.cuh"
#include "sh_codec.cuh"

namespace hg {

namespace {

constexpr int HIST_BINS = 4096;
constexpr float PERCENTILE = 0.995f;

__device__ __forceinline__ void ycocg(const float* c, float& y, float& co, float& cg) {
  co = __fsub_rn(c[0], c[2]);
  const float t = __fadd_rn(c[2], __fmul_rn(co, 0.5f));
  cg = __fsub_rn(c[1], t);
  y = __fadd_rn(t, __fmul_rn(cg, 0.5f));
}

// channel maxima of |Y|, |Co|, |Cg| (non-negative floats order as integers)
__global__ void k_codec_max(const float* sh, long long n, unsigned int* mx) {
  __shared__ unsigned int s_mx[SH_CODEC_CH];
  if (threadIdx.x < SH_CODEC_CH) s_mx[threadIdx.x] = 0;
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    for (int k = 0; k < SH_CODEC_BASES; ++k) {
      float v[3];
      ycocg(sh + (i * SH_CODEC_BASES + k) * 3, v[0], v[1], v[2]);
      for (int c = 0; c < 3; ++c) atomicMax(&s_mx[k * 3 + c], __float_as_uint(fabsf(v[c])));
    }
  }
  __syncthreads();
  if (threadIdx.x < SH_CODEC_CH) atomicMax(&mx[threadIdx.x], s_mx[threadIdx.x]);
}

__global__ void k_codec_hist(const float* sh, long long n, const unsigned int* mx, unsigned int* hist) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    for (int k = 0; k < SH_CODEC_BASES; ++k) {
      float v[3];
      ycocg(sh + (i * SH_CODEC_BASES + k) * 3, v[0], v[1], v[2]);
      for (int c = 0; c < 3; ++c) {
        const int ch = k * 3 + c;
        const float m = __uint_as_float(mx[ch]);
        const int b = m > 0.f ? min(HIST_BINS - 1, (int)(fabsf(v[c]) / m * HIST_BINS)) : 0;
        atomicAdd(&hist[ch * HIST_BINS + b], 1u);
      }
    }
  }
}

// one thread per channel: s = upper edge of the bin where the cumulative
// count reaches the percentile; s2 = s / Q^2 for the decoder
__global__ void k_codec_scales(long long n, const unsigned int* mx, const unsigned int* hist, float* scale,
                               float* scale2) {
  const int ch = threadIdx.x;
  if (ch >= SH_CODEC_CH) return;
  const float m = __uint_as_float(mx[ch]);
  const unsigned long long want = (unsigned long long)ceil((double)PERCENTILE * (double)n);
  unsigned long long cum = 0;
  int b = 0;
  for (; b < HIST_BINS; ++b) {
    cum += hist[ch * HIST_BINS + b];
    if (cum >= want) break;
  }
  float s = m > 0.f ? m * (float)(min(b, HIST_BINS - 1) + 1) / (float)HIST_BINS : 1.f;
  if (!(s > 0.f)) s = 1.f;
  const int bits = sh_codec_bits(ch / 3, ch % 3);
  const float q = (float)((1 << (bits - 1)) - 1);
  scale[ch] = s;
  scale2[ch] = ch < 3 ? s / (float)SH_CODEC_DC_Q : s / (q * q);
}

__global__ void k_codec_encode(const float* sh, long long n, const float* scale, uint32_t* codes) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < SH_CODEC_BASES; ++k) {
    float v[3];
    ycocg(sh + (i * SH_CODEC_BASES + k) * 3, v[0], v[1], v[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int bits = sh_codec_bits(k, c), pos = sh_codec_pos(k, c);
      uint32_t field;
      if (k == 0 && c == 0) {
        field = (uint32_t)__half_as_ushort(__float2half_rn(v[0]));
      } else {
        const float x = fminf(fmaxf(__fdiv_rn(v[c], scale[k * 3 + c]), -1.f), 1.f);
        int q;
        if (k == 0) {
          q = (int)rintf(__fmul_rn(x, (float)SH_CODEC_DC_Q));
        } else {
          const float qm = (float)((1 << (bits - 1)) - 1);
          q = (int)rintf(__fmul_rn(copysignf(__fsqrt_rn(fabsf(x)), x), qm));
        }
        field = (uint32_t)q & ((1u << bits) - 1u);
      }
      const int wi = pos >> 5, off = pos & 31;
      w[wi] |= field << off;
      if (off + bits > 32) w[wi + 1] |= field >> (32 - off);
    }
  }
  uint4* dst = reinterpret_cast<uint4*>(codes + i * 8);
  dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
  dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

}  // namespace

// Encodes n gaussians' degree-3 SH (device float32 [n][16][3]) into
// codes [n][8] and the per-channel scales (scale, scale / Q^2; device [48]).
hg_status sh_codec_encode(hg_ctx* ctx, const float* sh, long long n, uint32_t* codes, float* scale, float* scale2) {
  const size_t aux = sizeof(unsigned int) * SH_CODEC_CH * (1 + HIST_BINS);
  unsigned int* tmp = (unsigned int*)ctx_alloc(ctx, aux, nullptr);
  if (!tmp) return HG_ERR_OOM;
  unsigned int* mx = tmp;
  unsigned int* hist = tmp + SH_CODEC_CH;
  cudaError_t e = cudaMemset(tmp, 0, aux);
  const int grid = ctx->sms * 4;
  if (e == cudaSuccess && n > 0) {
    k_codec_max<<<grid, 256>>>(sh, n, mx);
    note_launch();
    k_codec_hist<<<grid, 256>>>(sh, n, mx, hist);
    note_launch();
  }
  if (e == cudaSuccess) {
    k_codec_scales<<<1, 64>>>(n, mx, hist, scale, scale2);
    note_launch();
  }
  if (e == cudaSuccess && n > 0) {
    k_codec_encode<<<(unsigned)((n + 127) / 128), 128>>>(sh, n, scale, codes);
    note_launch();
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  ctx_free(ctx, tmp, aux, nullptr);
  return e == cudaSuccess ? HG_OK : hg_cuda_status(e, "sh codec encode");
}

}  // namespace hg
