// Layout of the 32-byte packed SH representation (Sec. 4.2) and its
// decoder: 16 bases of degree-3 SH, each as (Y, Co, Cg) fields packed from
// bit 0 of word 0 of 8 uint32 words.  Bases 1..15: two's-complement fields
// of 6/4/4 bits, square-root gamma (a field q decodes to q |q| s / Q^2).
// Basis 0 (DC): Y as float16 bits (16), Co and Cg linear in 13 bits
// (q s / 4095).  Per channel the decoder keeps s / Q^2 (or s / 4095).
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"

namespace hg {

constexpr int SH_CODEC_BASES = 16;
constexpr int SH_CODEC_CH = 48;
constexpr int SH_CODEC_WORDS = 8;

constexpr int SH_CODEC_DC_Q = 4095;  // linear DC chroma levels

__host__ __device__ constexpr int sh_codec_bits(int k, int c) { return k == 0 ? (c == 0 ? 16 : 13) : (c == 0 ? 6 : 4); }

__host__ __device__ constexpr int sh_codec_pos(int k, int c) {
  return k == 0 ? (c == 0 ? 0 : (c == 1 ? 16 : 29)) : 42 + 14 * (k - 1) + (c == 0 ? 0 : (c == 1 ? 6 : 10));
}

// signed field (bits at position pos) of the 8 code words
template <int POS, int BITS>
__device__ __forceinline__ int sh_codec_field(const uint32_t* w) {
  constexpr int WI = POS >> 5, OFF = POS & 31;
  uint32_t v = w[WI] >> OFF;
  if (OFF + BITS > 32) v |= w[WI + 1] << (32 - OFF);
  return (int)(v << (32 - BITS)) >> (32 - BITS);
}

// RGB coefficients of basis K from the code words and s / Q^2 per channel
template <int K>
__device__ __forceinline__ void sh_codec_basis(const uint32_t* w, const float* scale2, float& r, float& g, float& b) {
  const int qy = sh_codec_field<sh_codec_pos(K, 0), sh_codec_bits(K, 0)>(w);
  const int qo = sh_codec_field<sh_codec_pos(K, 1), sh_codec_bits(K, 1)>(w);
  const int qg = sh_codec_field<sh_codec_pos(K, 2), sh_codec_bits(K, 2)>(w);
  float y, co, cg;
  if (K == 0) {
    y = __half2float(__ushort_as_half((unsigned short)(qy & 0xffff)));
    co = (float)qo * scale2[1];
    cg = (float)qg * scale2[2];
  } else {
    y = (float)(qy * abs(qy)) * scale2[K * 3 + 0];
    co = (float)(qo * abs(qo)) * scale2[K * 3 + 1];
    cg = (float)(qg * abs(qg)) * scale2[K * 3 + 2];
  }
  const float t = y - 0.5f * cg;
  g = cg + t;
  b = t - 0.5f * co;
  r = b + co;
}

hg_status sh_codec_encode(hg_ctx* ctx, const float* sh, long long n, uint32_t* codes, float* scale, float* scale2);

}  // namespace hg
