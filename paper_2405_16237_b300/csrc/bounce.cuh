// Secondary bounce rays from predicted hits (Sec. 7: at a returned
// intersection the path tracer samples the next direction), and the
// counter-based generator they draw from.
#pragma once
#include "nbvh_internal.cuh"

namespace nbvh {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two
// 32x32->64 multiplies with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Top 24 bits of a uint32 as a float in [0, 1) (exact).
__device__ __forceinline__ float u24(uint32_t x) { return static_cast<float>(x >> 8) * (1.0f / 16777216.0f); }

struct RayOut {
  float *ox, *oy, *oz, *dx, *dy, *dz, *tmin, *tmax;
};

constexpr float kBounceOffset = 1e-4f;
constexpr float kTwoPi = 6.28318530717958647692f;

// For a hit: origin o + t d + 1e-4 n' (n' the predicted normal turned to face
// -d), direction cosine-weighted about n' from Philox counter (ray, 0, 0, 2)
// with r = sqrt(u1), phi = 2 pi u2, expressed in the orthonormal basis of
// Duff et al. (JCGT 2017). A miss gets an empty interval (tmin 0, tmax -1).
static __global__ void __launch_bounds__(256) bounce_kernel(RayPtrs in, nbvh_hits hits, int64_t n, uint32_t k0,
                                                     uint32_t k1, RayOut out) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const float ox = in.ox[r], oy = in.oy[r], oz = in.oz[r];
  const float dx = in.dx[r], dy = in.dy[r], dz = in.dz[r];
  if (!hits.hit[r]) {
    out.ox[r] = ox; out.oy[r] = oy; out.oz[r] = oz;
    out.dx[r] = dx; out.dy[r] = dy; out.dz[r] = dz;
    out.tmin[r] = 0.0f;
    out.tmax[r] = -1.0f;
    return;
  }
  float nx = hits.nx[r], ny = hits.ny[r], nz = hits.nz[r];
  if (nx * dx + ny * dy + nz * dz > 0.0f) { nx = -nx; ny = -ny; nz = -nz; }
  const float t = hits.t[r];
  out.ox[r] = ox + t * dx + kBounceOffset * nx;
  out.oy[r] = oy + t * dy + kBounceOffset * ny;
  out.oz[r] = oz + t * dz + kBounceOffset * nz;
  const uint4 q = philox4x32_10(make_uint4(uint32_t(r), uint32_t(uint64_t(r) >> 32), 0u, 2u), k0, k1);
  const float u1 = u24(q.x), u2 = u24(q.y);
  const float rad = sqrtf(u1);
  float sp, cp;
  sincosf(kTwoPi * u2, &sp, &cp);
  const float lx = rad * cp, ly = rad * sp, lz = sqrtf(fmaxf(0.0f, 1.0f - u1));
  const float sgn = nz >= 0.0f ? 1.0f : -1.0f;
  const float a = -1.0f / (sgn + nz);
  const float b = nx * ny * a;
  const float tx = 1.0f + sgn * nx * nx * a, ty = sgn * b, tz = -sgn * nx;
  const float bx = b, by = sgn + ny * ny * a, bz = -ny;
  out.dx[r] = lx * tx + ly * bx + lz * nx;
  out.dy[r] = lx * ty + ly * by + lz * ny;
  out.dz[r] = lx * tz + ly * bz + lz * nz;
  out.tmin[r] = 0.0f;
  out.tmax[r] = __int_as_float(0x7f800000);
}

}  // namespace nbvh
