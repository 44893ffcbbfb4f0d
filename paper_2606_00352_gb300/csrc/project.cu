// Fused projection + SH colour front end (Sec. 4.2): one thread per gaussian
// handles every view of the frame, so the gaussian's attributes are read from
// HBM once per frame.  The CTA's contiguous slices of the five attribute
// arrays are staged into shared memory with TMA bulk copies.
//
// Outputs per (view, gaussian), index v * N + i:
//   bin  uint4  plain path: {mx bits, my bits, radius, depth key}; HiGS: the
//               binning record of the macro cells (binning.cuh), with the
//               depth key in dkeys
//   rec  float4 x4 {mx, my, l0', l1'} {l2', o, radius bits, key bits} {r, g, b, E''} {0}
//        (E'': the per-gaussian level of the blend test, blend_level)
//   vis  one bit per gaussian, written per warp (Sec. 4.2 visibility bitfield)
// bin and rec are written for visible entries only.
// l' are the Cholesky factors of the conic prescaled by sqrt(log2(e)/2), so the
// rasteriser evaluates alpha = o exp2(-((l0' dx + l1' dy)^2 + (l2' dy)^2)).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "binning.cuh"
#include "blend.cuh"
#include "kernels.cuh"
#include "sh_codec.cuh"

namespace hg {

namespace {

constexpr int PROJ_THREADS = 128;  // 7 CTAs per SM: more staged copies in flight than 3 x 256

__device__ __forceinline__ float sh_f(float x) { return x; }
__device__ __forceinline__ float sh_f(__half x) { return __half2float(x); }
__device__ __forceinline__ float sh_f(__nv_bfloat16 x) { return __bfloat162float(x); }

// Tag of the 32-byte packed SH representation (sh_codec.cuh).
struct ShCodec32 {};

// SH coefficients are staged in their storage form and converted when used
// (float32 arithmetic either way): PER elements of type T per gaussian.
template <int DEG, typename SHT>
struct ShStage {
  using T = SHT;
  static constexpr int PER = (DEG + 1) * (DEG + 1) * 3;
};
template <int DEG>
struct ShStage<DEG, ShCodec32> {
  using T = uint32_t;
  static constexpr int PER = SH_CODEC_WORDS;
};

template <int DEG, typename SHT>
struct ProjSmem {
  float means[PROJ_THREADS * 3];
  float scales[PROJ_THREADS * 3];
  float4 quats[PROJ_THREADS];
  float logits[PROJ_THREADS];
  alignas(16) typename ShStage<DEG, SHT>::T sh[PROJ_THREADS * ShStage<DEG, SHT>::PER];
  float sh_scale2[SH_CODEC_CH];  // packed SH: s / Q^2 per channel
  uint64_t bar;
  ViewDesc views[1];  // [n_views], sized at launch
};

// The coefficients of band L: converted from the staged type, or decoded
// from the 32-byte packed form.  When a gaussian's staged row (PER elements)
// is a multiple of 16 bytes (degree 3: float32 rows of 192 bytes, half rows
// of 96), a band is read as the 16-byte vectors that hold it: four times
// fewer shared loads than element loads, and with that row stride between
// threads, four times fewer bank conflicts.
template <typename T>
__device__ __forceinline__ T vec_elem(const uint4& v, int e) {
  return reinterpret_cast<const T*>(&v)[e];
}

template <int L, typename SHT, int PER>
struct BandLoad {
  template <typename T>
  __device__ static void run(const T* g, float* c, const float*) {
    constexpr int B = 2 * L + 1, OFF = L * L;
    if constexpr ((PER * sizeof(T)) % 16 == 0) {
      constexpr int E = 16 / (int)sizeof(T);  // elements per vector
      constexpr int V0 = OFF * 3 / E, V1 = ((OFF + B) * 3 - 1) / E;
      const uint4* g4 = reinterpret_cast<const uint4*>(g);
      uint4 v[V1 - V0 + 1];
#pragma unroll
      for (int i = 0; i <= V1 - V0; ++i) v[i] = g4[V0 + i];
#pragma unroll
      for (int k = 0; k < B * 3; ++k) c[k] = sh_f(vec_elem<T>(v[(OFF * 3 + k) / E - V0], (OFF * 3 + k) % E));
    } else {
#pragma unroll
      for (int k = 0; k < B * 3; ++k) c[k] = sh_f(g[OFF * 3 + k]);
    }
  }
};

template <int K0, int N>
__device__ __forceinline__ void codec_bases(const uint32_t* w, const float* s2, float* c) {
  if constexpr (N > 0) {
    sh_codec_basis<K0>(w, s2, c[0], c[1], c[2]);
    codec_bases<K0 + 1, N - 1>(w, s2, c + 3);
  }
}

template <int L, int PER>
struct BandLoad<L, ShCodec32, PER> {
  __device__ static void run(const uint32_t* w, float* c, const float* s2) {
    codec_bases<L * L, 2 * L + 1>(w, s2, c);
  }
};

template <int DEG, typename SHT>
__host__ __device__ constexpr size_t proj_smem_bytes(int n_views) {
  return sizeof(ProjSmem<DEG, SHT>) + sizeof(ViewDesc) * (size_t)(n_views > 1 ? n_views - 1 : 0);
}

// SH colour of one band for up to VG views: acc[v] += sum_m Y_lm(d_v) c_lm.
template <int L, int VG, typename SHT, int PER, typename T>
__device__ __forceinline__ void sh_band(const T* __restrict__ sh_g, const float (&d)[VG][3], float (&acc)[VG][3],
                                        int nv, const float* s2) {
  constexpr int B = 2 * L + 1;
  float c[B * 3];
  BandLoad<L, SHT, PER>::run(sh_g, c, s2);
#pragma unroll
  for (int v = 0; v < VG; ++v) {
    if (v >= nv) break;
    const float x = d[v][0], y = d[v][1], z = d[v][2];
    float Y[B];
    if (L == 0) {
      Y[0] = 0.28209479177387814f;  // 1/(2 sqrt(pi))
    } else if (L == 1) {
      const float C1 = 0.48860251190291992f;  // sqrt(3/(4 pi))
      Y[0] = -C1 * y;
      Y[1] = C1 * z;
      Y[2] = -C1 * x;
    } else if (L == 2) {
      const float C2a = 1.0925484305920792f;   // (1/2) sqrt(15/pi)
      const float C2b = 0.31539156525252005f;  // (1/4) sqrt(5/pi)
      const float C2c = 0.54627421529603959f;  // (1/4) sqrt(15/pi)
      const float xx = x * x, yy = y * y, zz = z * z;
      Y[0] = C2a * x * y;
      Y[1] = -C2a * y * z;
      Y[2] = C2b * (2.f * zz - xx - yy);
      Y[3] = -C2a * x * z;
      Y[4] = C2c * (xx - yy);
    } else {
      const float C3a = 0.59004358992664352f;  // (1/4) sqrt(35/(2 pi))
      const float C3b = 2.8906114426405538f;   // (1/2) sqrt(105/pi)
      const float C3c = 0.45704579946446577f;  // (1/4) sqrt(21/(2 pi))
      const float C3d = 0.3731763325901154f;   // (1/4) sqrt(7/pi)
      const float C3e = 1.4453057213202769f;   // (1/4) sqrt(105/pi)
      const float xx = x * x, yy = y * y, zz = z * z;
      const float t4 = 4.f * zz - xx - yy;
      Y[0] = -C3a * y * (3.f * xx - yy);
      Y[1] = C3b * x * y * z;
      Y[2] = -C3c * y * t4;
      Y[3] = C3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[4] = -C3c * x * t4;
      Y[5] = C3e * z * (xx - yy);
      Y[6] = -C3a * x * (xx - 3.f * yy);
    }
#pragma unroll
    for (int m = 0; m < B; ++m) {
      acc[v][0] = fmaf(Y[m], c[3 * m + 0], acc[v][0]);
      acc[v][1] = fmaf(Y[m], c[3 * m + 1], acc[v][1]);
      acc[v][2] = fmaf(Y[m], c[3 * m + 2], acc[v][2]);
    }
  }
}

// One thread per gaussian, every view of the frame.  Two passes per thread
// keep the register footprint small (more CTAs per SM, so more copies in
// flight): geometry for every view (bin record and the first 32 bytes of the
// raster record), then the SH colour band by band for groups of up to 4
// views, each band's coefficients read from shared memory once per group.
// Culled (view, gaussian) entries write nothing: consumers test the
// visibility bits first.
template <int DEG, typename SHT>
__global__ void __launch_bounds__(PROJ_THREADS) k_project(ProjectArgs a) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int VG = 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ProjSmem<DEG, SHT>& s = *reinterpret_cast<ProjSmem<DEG, SHT>*>(smem_raw);
  using ST = typename ShStage<DEG, SHT>::T;
  constexpr int PER = ShStage<DEG, SHT>::PER;
  const ST* sh_in = reinterpret_cast<const ST*>(a.sh);
  const int tid = threadIdx.x;
  const long long i0 = (long long)blockIdx.x * PROJ_THREADS;
  const int cnt = (int)min((long long)PROJ_THREADS, a.n - i0);
  const bool full = cnt == PROJ_THREADS;
  const int nv = a.n_views;
  // visible-entry count of the CTA: one global atomic per CTA (a counter
  // updated by every warp and view serialises at its L2 slice)
  __shared__ uint32_t s_nvis, s_warps_done;
  if (tid == 0) s_nvis = s_warps_done = 0;

  if (full) {
    // TMA: five contiguous slices, one mbarrier
    if (tid == 0) {
      mbar_init(&s.bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
      const uint32_t b3 = PROJ_THREADS * 12, b4 = PROJ_THREADS * 16, b1 = PROJ_THREADS * 4,
                     bsh = PROJ_THREADS * PER * (uint32_t)sizeof(ST);
      mbar_arrive_expect_tx(&s.bar, 2 * b3 + b4 + b1 + bsh);
      tma_load_1d(s.means, a.means + i0 * 3, b3, &s.bar);
      tma_load_1d(s.scales, a.log_scales + i0 * 3, b3, &s.bar);
      tma_load_1d(s.quats, a.quats + i0 * 4, b4, &s.bar);
      tma_load_1d(s.logits, a.opacity_logits + i0, b1, &s.bar);
      tma_load_1d(s.sh, sh_in + i0 * PER, bsh, &s.bar);
    }
  } else {
    for (int j = tid; j < cnt * 3; j += PROJ_THREADS) {
      s.means[j] = a.means[i0 * 3 + j];
      s.scales[j] = a.log_scales[i0 * 3 + j];
    }
    for (int j = tid; j < cnt; j += PROJ_THREADS) {
      s.quats[j] = reinterpret_cast<const float4*>(a.quats)[i0 + j];
      s.logits[j] = a.opacity_logits[i0 + j];
    }
    for (int j = tid; j < cnt * PER; j += PROJ_THREADS) s.sh[j] = sh_in[i0 * PER + j];
  }
  // the view table (and the packed-SH scales), while the copies are in flight
  if (a.sh_scale2 && tid < SH_CODEC_CH) s.sh_scale2[tid] = a.sh_scale2[tid];
  {
    const int words = nv * (int)(sizeof(ViewDesc) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.views);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s.views);
    for (int j = tid; j < words; j += PROJ_THREADS) dst[j] = src[j];
  }
  if (full && !mbar_wait_bounded(&s.bar, 0, a.wait_polls)) {
    set_status(a.fc, HG_ERR_DEVICE_TIMEOUT);
    atomicOr(&a.fc->timeout_where, 4u);
    // the copies were issued by this CTA: wait (bounded again) before exit
    mbar_wait_bounded(&s.bar, 0);
    return;
  }
  __syncthreads();

  const bool valid = tid < cnt;
  const long long gi = i0 + tid;
  const int lane = tid & 31;
  float px = 0.f, py = 0.f, pz = 0.f, op = 0.f;
  unsigned long long vbits = 0;  // views in which the gaussian is visible
  uint32_t warp_vis = 0;         // lane 0: visible entries of the warp
  {
    float sx = 1.f, sy = 1.f, sz = 1.f;
    float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
    if (valid) {
      px = s.means[tid * 3 + 0];
      py = s.means[tid * 3 + 1];
      pz = s.means[tid * 3 + 2];
      sx = __expf(s.scales[tid * 3 + 0]);
      sy = __expf(s.scales[tid * 3 + 1]);
      sz = __expf(s.scales[tid * 3 + 2]);
      q = s.quats[tid];
      op = __fdividef(1.f, 1.f + __expf(-s.logits[tid]));
    }
    // rotation of the normalised quaternion (w, x, y, z), times the scales
    const float qn = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * qn, x = q.y * qn, y = q.z * qn, z = q.w * qn;
    const float M[3][3] = {
        {(1.f - 2.f * (y * y + z * z)) * sx, 2.f * (x * y - w * z) * sy, 2.f * (x * z + w * y) * sz},
        {2.f * (x * y + w * z) * sx, (1.f - 2.f * (x * x + z * z)) * sy, 2.f * (y * z - w * x) * sz},
        {2.f * (x * z - w * y) * sx, 2.f * (y * z + w * x) * sy, (1.f - 2.f * (x * x + y * y)) * sz}};

    for (int v = 0; v < nv; ++v) {
      const ViewDesc& V = s.views[v];
      // depth in the pinned float32 order (no contraction): the sort key
      const float tz = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(V.vm[8], px), __fmul_rn(V.vm[9], py)),
                                           __fmul_rn(V.vm[10], pz)),
                                 V.vm[11]);
      const float tx = fmaf(V.vm[0], px, fmaf(V.vm[1], py, fmaf(V.vm[2], pz, V.vm[3])));
      const float ty = fmaf(V.vm[4], px, fmaf(V.vm[5], py, fmaf(V.vm[6], pz, V.vm[7])));
      bool vis = valid && tz > 0.2f;
      const float itz = __fdividef(1.f, tz);
      const float limx = 1.3f * V.tan_x, limy = 1.3f * V.tan_y;
      const float ux = fminf(fmaxf(tx * itz, -limx), limx);
      const float uy = fminf(fmaxf(ty * itz, -limy), limy);
      const float j00 = V.fx * itz, j02 = -V.fx * ux * itz;
      const float j11 = V.fy * itz, j12 = -V.fy * uy * itz;
      // T = J W (2x3), then TM = T M
      float t0[3], t1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        t0[k] = fmaf(j00, V.vm[k], j02 * V.vm[8 + k]);
        t1[k] = fmaf(j11, V.vm[4 + k], j12 * V.vm[8 + k]);
      }
      float m0[3], m1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        m0[k] = fmaf(t0[0], M[0][k], fmaf(t0[1], M[1][k], t0[2] * M[2][k]));
        m1[k] = fmaf(t1[0], M[0][k], fmaf(t1[1], M[1][k], t1[2] * M[2][k]));
      }
      const float ca = fmaf(m0[0], m0[0], fmaf(m0[1], m0[1], m0[2] * m0[2])) + 0.3f;
      const float cb = fmaf(m0[0], m1[0], fmaf(m0[1], m1[1], m0[2] * m1[2]));
      const float cc = fmaf(m1[0], m1[0], fmaf(m1[1], m1[1], m1[2] * m1[2])) + 0.3f;
      const float det = ca * cc - cb * cb;
      vis = vis && det > 0.f;
      const float mid = 0.5f * (ca + cc);
      const float dq = fmaxf(0.1f, mid * mid - det);
      const float lam = mid + dq * rsqrtf(dq);
      const float rr = ceilf(3.f * (lam * rsqrtf(lam)));
      int rad = (int)fminf(rr, (float)RADIUS_MAX);
      const float mx = fmaf(V.fx, tx * itz, V.cx - 0.5f);
      const float my = fmaf(V.fy, ty * itz, V.cy - 0.5f);
      vis = vis && rad > 0 && fabsf(mx) < 1e7f && fabsf(my) < 1e7f;
      if (vis) {
        const int x0 = (int)floorf(mx), y0 = (int)floorf(my);
        vis = (x0 + rad >= 0) && (x0 - rad <= V.W - 1) && (y0 + rad >= 0) && (y0 - rad <= V.H - 1);
      }
      if (!vis) rad = 0;
      // Cholesky of the conic: l0 = sqrt(c/det), l1 = -b / sqrt(c det), l2 = 1/sqrt(c)
      const float rc = rsqrtf(cc), rd = rsqrtf(det);
      const float l0 = cc * rc * rd * CHOL_PRESCALE;
      const float l1 = -cb * rc * rd * CHOL_PRESCALE;
      const float l2 = rc * CHOL_PRESCALE;
      const uint32_t key = __float_as_uint(tz);
      const long long o = (long long)v * a.n + gi;
      const uint32_t ballot = __ballot_sync(0xffffffffu, vis);
      if (vis) {
        vbits |= 1ull << v;
        if (a.bin_mode == BIN_CLASSIC) {
          a.bin[o] = make_uint4(__float_as_uint(mx), __float_as_uint(my), (uint32_t)rad, key);
        } else {
          a.bin[o] = bin_cells(mx, my, rad, l0, l1, l2, op, a.macro_w * TILE, a.macro_h * TILE, V.mgx, V.mgy,
                               a.bin_mode == BIN_CELLS_ELLIPSE);
          a.dkeys[o] = key;
        }
        float4* r = a.rec + o * REC_F4;
        r[0] = make_float4(mx, my, l0, l1);
        r[1] = make_float4(l2, op, __int_as_float(rad), __uint_as_float(key));
      }
      if (a.splats && valid) {
        hg_splat sp;
        const float idet = 1.f / det;
        sp.mean2d[0] = mx;
        sp.mean2d[1] = my;
        sp.conic[0] = cc * idet;
        sp.conic[1] = -cb * idet;
        sp.conic[2] = ca * idet;
        sp.opacity = op;
        sp.rgb[0] = sp.rgb[1] = sp.rgb[2] = 0.f;  // the colour pass fills these
        sp.depth_key = key;
        sp.radius = rad;
        sp.depth = tz;
        a.splats[o] = sp;
      }
      if (lane == 0) {
        const long long word = (long long)v * a.vis_words + (gi >> 5);
        if (i0 + (tid & ~31) < a.n) a.vis[word] = ballot;
        warp_vis += (uint32_t)__popc(ballot);
      }
    }
  }
  if (lane == 0) {
    if (warp_vis) atomicAdd(&s_nvis, warp_vis);
    __threadfence_block();
    if (atomicAdd(&s_warps_done, 1u) == PROJ_THREADS / 32 - 1) {
      const uint32_t total = atomicAdd(&s_nvis, 0u);
      if (total) atomicAdd(&a.fc->n_visible, total);
    }
  }

  // view-dependent colour: max(0, SH(d) + 0.5), d = normalise(mean - campos)
  const ST* sh_g = s.sh + tid * PER;
  const bool keep = a.splats != nullptr && valid;
  for (int v0 = 0; v0 < nv; v0 += VG) {
    const int g = min(VG, nv - v0);
    const bool any = (vbits >> v0) & ((1ull << g) - 1ull);
    if (!__any_sync(0xffffffffu, any || keep)) continue;
    float d[VG][3], acc[VG][3];
#pragma unroll
    for (int v = 0; v < VG; ++v) {
      const ViewDesc& V = s.views[v0 + (v < g ? v : 0)];
      const float dx = px - V.campos[0], dy = py - V.campos[1], dz = pz - V.campos[2];
      const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
      d[v][0] = dx * dn;
      d[v][1] = dy * dn;
      d[v][2] = dz * dn;
      acc[v][0] = acc[v][1] = acc[v][2] = 0.f;
    }
    sh_band<0, VG, SHT, PER>(sh_g, d, acc, g, s.sh_scale2);
    if (DEG >= 1) sh_band<1, VG, SHT, PER>(sh_g, d, acc, g, s.sh_scale2);
    if (DEG >= 2) sh_band<2, VG, SHT, PER>(sh_g, d, acc, g, s.sh_scale2);
    if (DEG >= 3) sh_band<3, VG, SHT, PER>(sh_g, d, acc, g, s.sh_scale2);
#pragma unroll
    for (int v = 0; v < VG; ++v) {
      if (v >= g) break;
      const float cr = fmaxf(acc[v][0] + 0.5f, 0.f);
      const float cg = fmaxf(acc[v][1] + 0.5f, 0.f);
      const float cbl = fmaxf(acc[v][2] + 0.5f, 0.f);
      const long long o = (long long)(v0 + v) * a.n + gi;
      if ((vbits >> (v0 + v)) & 1ull) {
        a.rec[o * REC_F4 + 2] = make_float4(cr, cg, cbl, blend_level(op));
        a.rec[o * REC_F4 + 3] = make_float4(0.f, 0.f, 0.f, 0.f);  // stride padding (whole 64-byte writes)
      }
      if (keep) {
        a.splats[o].rgb[0] = cr;
        a.splats[o].rgb[1] = cg;
        a.splats[o].rgb[2] = cbl;
      }
    }
  }
}

// Public splat records -> internal records (used by hg_render_splats).
__global__ void k_splats_to_records(const hg_splat* sp, long long total, long long n, ProjectArgs out) {
  long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = o < total;
  hg_splat s;
  bool on = false;
  if (valid) {
    s = sp[o];
    const long long v = o / n;
    const ViewDesc& V = out.views[v];
    on = s.radius > 0 && fabsf(s.mean2d[0]) < 1e7f && fabsf(s.mean2d[1]) < 1e7f;
    // Cholesky factors, each operation rounded as written (reproducible)
    const float l0 = __fsqrt_rn(fmaxf(s.conic[0], 0.f));
    const float l1 = l0 > 0.f ? __fdiv_rn(s.conic[1], l0) : 0.f;
    const float l2 = __fsqrt_rn(fmaxf(__fsub_rn(s.conic[2], __fmul_rn(l1, l1)), 0.f));
    const float L0 = __fmul_rn(l0, CHOL_PRESCALE), L1 = __fmul_rn(l1, CHOL_PRESCALE), L2 = __fmul_rn(l2, CHOL_PRESCALE);
    const int rad = on ? min(s.radius, RADIUS_MAX) : 0;
    if (out.bin_mode == BIN_CLASSIC)
      out.bin[o] = make_uint4(__float_as_uint(s.mean2d[0]), __float_as_uint(s.mean2d[1]), (uint32_t)rad, s.depth_key);
    else
      out.bin[o] = bin_cells(s.mean2d[0], s.mean2d[1], rad, L0, L1, L2, s.opacity, out.macro_w * TILE,
                             out.macro_h * TILE, V.mgx, V.mgy, out.bin_mode == BIN_CELLS_ELLIPSE);
    out.dkeys[o] = s.depth_key;
    out.rec[o * REC_F4 + 0] = make_float4(s.mean2d[0], s.mean2d[1], L0, L1);
    out.rec[o * REC_F4 + 1] = make_float4(L2, s.opacity, __int_as_float(rad), __uint_as_float(s.depth_key));
    out.rec[o * REC_F4 + 2] = make_float4(s.rgb[0], s.rgb[1], s.rgb[2], blend_level(s.opacity));
    out.rec[o * REC_F4 + 3] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // visibility words: the splat array is [V][n]; a warp's 32 entries map to
  // one word only when n is a multiple of 32, so set bits atomically.
  if (valid && on) {
    long long v = o / n, i = o % n;
    atomicOr(&out.vis[v * out.vis_words + (i >> 5)], 1u << (i & 31));
  }
}

}  // namespace

template <int DEG, typename SHT>
static cudaError_t launch_project_t(const ProjectArgs& a, cudaStream_t st) {
  size_t sm = proj_smem_bytes<DEG, SHT>(a.n_views);
  cudaError_t e = cudaFuncSetAttribute(k_project<DEG, SHT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  long long blocks = (a.n + PROJ_THREADS - 1) / PROJ_THREADS;
  if (blocks == 0) return cudaSuccess;
  k_project<DEG, SHT><<<(unsigned)blocks, PROJ_THREADS, sm, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <int DEG>
static cudaError_t launch_project_deg(const ProjectArgs& a, cudaStream_t st) {
  switch (a.sh_storage) {
    case HG_SH_F16: return launch_project_t<DEG, __half>(a, st);
    case HG_SH_BF16: return launch_project_t<DEG, __nv_bfloat16>(a, st);
    case HG_SH_CODEC32:
      if (DEG != 3) return cudaErrorInvalidValue;
      return launch_project_t<DEG, ShCodec32>(a, st);
    default: return launch_project_t<DEG, float>(a, st);
  }
}

cudaError_t launch_project(const ProjectArgs& a, int deg, cudaStream_t st) {
  switch (deg) {
    case 0: return launch_project_deg<0>(a, st);
    case 1: return launch_project_deg<1>(a, st);
    case 2: return launch_project_deg<2>(a, st);
    default: return launch_project_deg<3>(a, st);
  }
}

cudaError_t launch_splats_to_records(const hg_splat* sp, long long n, int n_views, long long vis_words,
                                     const ProjectArgs& out, cudaStream_t st) {
  long long total = n * n_views;
  cudaError_t e = cudaMemsetAsync(out.vis, 0, sizeof(uint32_t) * vis_words * n_views, st);
  if (e != cudaSuccess || total == 0) return e;
  k_splats_to_records<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(sp, total, n, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace hg
