// 3-D implicit-step operators for n_f order parameters (Fan-Chen grain growth
// or the double well), JAX-PF Eq. 13-14:
//   R(U) = M (U - U^n)/dt + L r(U),     J v = M v / dt + L H(U) v,
// with r the gradient and H the Hessian of E_h = sum_e sum_q w|J| [f(U_q) +
// kappa/2 |grad U_q|^2].  Both are evaluated scaled by the lumped mass,
// G = M^-1 R and M^-1 J v, on a mirror-extended tile: the mirror images of
// boundary elements double the partial sums exactly where the lumped mass
// halves, so every node uses the interior formula (an optional final
// multiplication by m_i gives R and J v themselves).
//
// Work split: 16 x 8 node columns in x, y; one wave of resident blocks, each
// sweeping an equal share of the column planes along z (the kernel below
// describes the steps).  One thread per (element, field pair) forms the
// trilinear Gauss values (sum-factorised), the pointwise f' or H v, and the
// gradient term kappa grad w . grad N_a (w = U for the residual, v for the
// JVP), weighted back to the 8 corners; the lanes of an element sum the field
// couplings S2 = sum_f U_f^2 and T = sum_f U_f v_f by warp shuffles; a
// node-centric gather adds the 8 element contributions and the mass term.
// The gradient term needs no extra loads: the three passes of the
// sum-factorised interpolation already form the element's differences along
// x, y and z, which (interpolated in the other directions) are the Gauss-point
// derivatives; their weights back enter the matching passes of the projection.
// 2x2x2 Gauss integrates the Q1 stiffness exactly, so this is the assembled
// 27-point stencil, evaluated element by element on differences.
// Fields travel in pairs: shared memory holds (field 2p, field 2p+1) side by
// side (a zero field pads an odd count), one 64-bit load fetches both, and
// every interpolation, pointwise term, projection and stencil runs on packed
// FP32 pairs with the f32x2 instructions of sm_100+.
// No atomics: the gather order is fixed, so results are bitwise repeatable.
#include <algorithm>

#include "pf_internal.h"

namespace pf {
namespace {

typedef unsigned long long u64;  // packed FP32 pair: low half = the even field

__device__ __forceinline__ u64 pk(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float plo(u64 v) {
  float l;
  asm("{ .reg .f32 t; mov.b64 {%0, t}, %1; }" : "=f"(l) : "l"(v));
  return l;
}
__device__ __forceinline__ float phi(u64 v) {
  float h;
  asm("{ .reg .f32 t; mov.b64 {t, %0}, %1; }" : "=f"(h) : "l"(v));
  return h;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 bc(float v) { return pk(v, v); }

// Single mirror image about the end nodes, then clamped into the mesh: exact
// for the 1-node halo of stored nodes when the mesh has at least 2 nodes;
// positions further out (the far side of a ragged last tile) only feed
// outputs that are not stored, and the clamp keeps their loads in bounds.
__device__ __forceinline__ int reflect(int k, int n) {
  k = k < 0 ? -k : k;
  k = k >= n ? 2 * (n - 1) - k : k;
  return k < 0 ? 0 : (k >= n ? n - 1 : k);
}


// values at the two Gauss points of a segment from its end values
__device__ __forceinline__ void interp1(u64 a, u64 b, u64& lo, u64& hi) {
  const u64 d = sub2(b, a);
  lo = fma2(bc(kGLo), d, a);
  hi = fma2(bc(kGHi), d, a);
}

// weights back: contributions of the two Gauss values to the segment's ends
__device__ __forceinline__ void project1(u64 lo, u64 hi, u64& a, u64& b) {
  const u64 d = sub2(hi, lo);
  a = fma2(bc(kGLo), d, lo);   // g_hi lo + g_lo hi
  b = fma2(bc(-kGLo), d, hi);  // g_lo lo + g_hi hi
}

// 8 corner values c[z][y][x] -> 8 Gauss values q[z][y][x] (tensor product)
__device__ __forceinline__ void interp3(const u64 c[8], u64 q[8]) {
  u64 t[8], u[8];
#pragma unroll
  for (int zy = 0; zy < 4; ++zy) interp1(c[2 * zy], c[2 * zy + 1], t[2 * zy], t[2 * zy + 1]);
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) interp1(t[4 * z + x], t[4 * z + 2 + x], u[4 * z + x], u[4 * z + 2 + x]);
#pragma unroll
  for (int yx = 0; yx < 4; ++yx) interp1(u[yx], u[4 + yx], q[yx], q[4 + yx]);
}

// interp3 plus the Gauss-point derivatives in local coordinates (one unit
// per element edge): gx[qz][qy] = d/dx (constant along x), gy[qz][qx],
// gz[qy][qx], each formed from the differences the passes already take
__device__ __forceinline__ void interp3_grad(const u64 c[8], u64 q[8], u64 gx[4], u64 gy[4],
                                             u64 gz[4]) {
  u64 t[8], u[8], d1[4], d2[4];
#pragma unroll
  for (int zy = 0; zy < 4; ++zy) {  // x pass: d1[zy] = x-difference on edge (y, z)
    d1[zy] = sub2(c[2 * zy + 1], c[2 * zy]);
    t[2 * zy] = fma2(bc(kGLo), d1[zy], c[2 * zy]);
    t[2 * zy + 1] = fma2(bc(kGHi), d1[zy], c[2 * zy]);
  }
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) {  // y pass: d2[2z + x] = y-difference at (qx = x, z)
      const u64 a = t[4 * z + x];
      d2[2 * z + x] = sub2(t[4 * z + 2 + x], a);
      u[4 * z + x] = fma2(bc(kGLo), d2[2 * z + x], a);
      u[4 * z + 2 + x] = fma2(bc(kGHi), d2[2 * z + x], a);
    }
#pragma unroll
  for (int yx = 0; yx < 4; ++yx) {  // z pass: its differences are d/dz at (qy, qx)
    gz[yx] = sub2(u[4 + yx], u[yx]);
    q[yx] = fma2(bc(kGLo), gz[yx], u[yx]);
    q[4 + yx] = fma2(bc(kGHi), gz[yx], u[yx]);
  }
  // d/dy at (qz, qx): d2 interpolated along z
#pragma unroll
  for (int x = 0; x < 2; ++x) interp1(d2[x], d2[2 + x], gy[x], gy[2 + x]);
  // d/dx at (qz, qy): d1[y + 2z] interpolated along y, then z
  u64 e[4];
#pragma unroll
  for (int z = 0; z < 2; ++z) interp1(d1[2 * z], d1[2 * z + 1], e[2 * z], e[2 * z + 1]);
#pragma unroll
  for (int y = 0; y < 2; ++y) interp1(e[y], e[2 + y], gx[y], gx[2 + y]);
}

// transpose of interp3 (Gauss values -> corner contributions) plus the
// gradient term sum_q grad w . grad N_a with per-axis weights k[d] = 2 kappa / h_d^2
// (the factor 2 sums the two Gauss points along the derivative's own axis,
// where the derivative is constant).  Each derivative enters the projection
// after the pass along its own axis, with the sign of N_a' on that axis.
__device__ __forceinline__ void project3_grad(const u64 q[8], const u64 gx[4], const u64 gy[4],
                                              const u64 gz[4], const float k[3], u64 c[8]) {
  u64 t[8], u[8];
#pragma unroll
  for (int yx = 0; yx < 4; ++yx) {  // z pass; t[4 az + yx]
    project1(q[yx], q[4 + yx], t[yx], t[4 + yx]);
    t[yx] = fma2(bc(-k[2]), gz[yx], t[yx]);
    t[4 + yx] = fma2(bc(k[2]), gz[yx], t[4 + yx]);
  }
  u64 py[4];  // d/dy weighted back along z: py[2 az + qx]
#pragma unroll
  for (int x = 0; x < 2; ++x) project1(gy[x], gy[2 + x], py[x], py[2 + x]);
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) {  // y pass; u[4 az + 2 ay + qx]
      project1(t[4 * z + x], t[4 * z + 2 + x], u[4 * z + x], u[4 * z + 2 + x]);
      u[4 * z + x] = fma2(bc(-k[1]), py[2 * z + x], u[4 * z + x]);
      u[4 * z + 2 + x] = fma2(bc(k[1]), py[2 * z + x], u[4 * z + 2 + x]);
    }
  u64 e[4], px[4];  // d/dx weighted back along y, then z: px[2 az + ay]
#pragma unroll
  for (int z = 0; z < 2; ++z) project1(gx[2 * z], gx[2 * z + 1], e[2 * z], e[2 * z + 1]);
#pragma unroll
  for (int y = 0; y < 2; ++y) project1(e[y], e[2 + y], px[y], px[2 + y]);
#pragma unroll
  for (int zy = 0; zy < 4; ++zy) {  // x pass; c[2 zy + ax]
    project1(u[2 * zy], u[2 * zy + 1], c[2 * zy], c[2 * zy + 1]);
    c[2 * zy] = fma2(bc(-k[0]), px[zy], c[2 * zy]);
    c[2 * zy + 1] = fma2(bc(k[0]), px[zy], c[2 * zy + 1]);
  }
}

// ---------------------------------------------------------------------------
// R and J v on column tiles that sweep along z.  The column planes (kSX x kSY
// output nodes of one node plane) are numbered column by column, and each
// resident block takes an equal contiguous range of them: one or two
// segments of a column.  Along a segment it walks the element layers from
// the one below its first plane to the last one inside it:
//   - node plane z+1 of U and v or U^n (fields in pairs, the kSNX x kSNY nodes
//     around the tile, mirrored at the mesh boundary) enters a 4-plane ring
//     in shared memory, pair index fastest, from registers loaded while the
//     previous layer computed;
//   - one thread per (element, field pair) interpolates U (and v for the JVP)
//     at the 8 Gauss points from its 8 corners, with the gradient of the
//     field the gradient term acts on, and the G threads of an element
//     (adjacent lanes, one per pair) sum S2 = sum_f U_f^2 (and T =
//     sum_f U_f v_f) by warp shuffles: every coupling of Eq. 13-14 is formed
//     from one interpolation per field, with no second pass;
//   - f' (or H v) and the gradient term are weighted back to the corners: the 4 on
//     the layer's lower face into a 2-layer ring, the 4 on its upper face into
//     a 3-layer ring;
//   - node plane z gathers its 8 element contributions (lower faces of layer
//     z, upper faces of layer z-1) in the fixed corner order, adds the mass
//     term and writes R or J v.
// One block barrier per layer: the gather of a plane and the element work of
// the next layer run in the same phase, the rings keeping what one writes
// apart from what the other reads.  No atomics, so results are bitwise
// repeatable.
#ifndef PF_SWEEP_SX
#define PF_SWEEP_SX 16
#endif
#ifndef PF_SWEEP_SY
#define PF_SWEEP_SY 8
#endif
#ifndef PF_SWEEP_MINB
#define PF_SWEEP_MINB 1
#endif
constexpr int kSX = PF_SWEEP_SX, kSY = PF_SWEEP_SY;  // output nodes per column tile in x, y
constexpr int kSNX = kSX + 2, kSNY = kSY + 2;    // staged nodes per plane
constexpr int kSEX = kSX + 1, kSEY = kSY + 1;    // elements per layer touching the tile
constexpr int kSPlane = kSNX * kSNY;
constexpr int kSElems = kSEX * kSEY;

template <int NP>
struct SweepCfg {
  static constexpr int G = NP >= 3 ? 4 : NP;  // lanes per element, one per field pair
  static constexpr int kThreads = (kSElems * G + 31) / 32 * 32;
  static constexpr int kItems = (kSPlane * NP + kThreads - 1) / kThreads;  // staged pairs per thread
  static constexpr size_t kSmem = sizeof(u64) * (size_t)NP * (2 * 4 * kSPlane + 8 * kSElems + 12 * kSElems);
};

template <int NF, bool kJVP>
__global__ void __launch_bounds__(SweepCfg<(NF + 1) / 2>::kThreads, PF_SWEEP_MINB)
    k_implicit3d_sweep(const Implicit3DArgs a) {
  constexpr int NP = (NF + 1) / 2;
  constexpr int G = SweepCfg<NP>::G, kThreads = SweepCfg<NP>::kThreads;
  constexpr int kItems = SweepCfg<NP>::kItems;
  extern __shared__ u64 smem[];
  u64* sU = smem;                        // [4 planes][kSPlane nodes][NP]
  u64* sW = sU + 4 * kSPlane * NP;       // v (JVP) or U^n (residual), same layout
  u64* sLowB = sW + 4 * kSPlane * NP;    // [2 layers][4 lower corners][kSElems][NP]
  u64* sUpB = sLowB + 8 * kSElems * NP;  // [3 layers][4 upper corners][kSElems][NP]

  const int tiles_x = (a.nx + kSX - 1) / kSX, tiles_y = (a.ny + kSY - 1) / kSY;
  const int64_t N = (int64_t)a.nx * a.ny * a.nz;
  const int64_t plane = (int64_t)a.nx * a.ny;
  const int tid = threadIdx.x;
  // this block's share of the column planes (column-major: all planes of
  // column 0, then column 1, ...), an equal contiguous range per block
  const int64_t total = (int64_t)tiles_x * tiles_y * a.nz;
  const int64_t g_end = total * (blockIdx.x + 1) / gridDim.x;
  int64_t ioff[kItems];
  int islot[kItems];
  u64 pu[kItems], pw[kItems];
  for (int64_t g = total * blockIdx.x / gridDim.x; g < g_end;) {
  // one segment: column col, output planes z0 .. z0 + cz - 1
  const int64_t col = g / a.nz;
  const int z0 = (int)(g % a.nz);
  const int cz = (int)min((int64_t)(a.nz - z0), g_end - g);
  g += cz;
  const int x0 = (int)(col % tiles_x) * kSX, y0 = (int)(col / tiles_x) * kSY;
  __syncthreads();  // the last segment's gather has finished with the shared buffers

  // staged items of this thread: node (in the plane) and pair, as global
  // offsets within a plane and field offsets
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int it = tid + k * kThreads;
    islot[k] = it < kSPlane * NP ? it : -1;
    const int node = it / NP;
    const int lx = node % kSNX, ly = node / kSNX;
    const int gx = reflect(x0 - 1 + lx, a.nx), gy = reflect(y0 - 1 + ly, a.ny);
    ioff[k] = (int64_t)gy * a.nx + gx;
  }
  auto fetch = [&](int z) {  // plane z (mirrored) of this thread's items into registers
    const int64_t zo = (int64_t)reflect(z, a.nz) * plane;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      pu[k] = pw[k] = 0;
      if (islot[k] >= 0) {
        const int p = islot[k] % NP;
        const int64_t g = zo + ioff[k];
        const int64_t f0 = (int64_t)(2 * p) * N + g;
        pu[k] = pk(__ldg(a.U + f0), 2 * p + 1 < NF ? __ldg(a.U + f0 + N) : 0.0f);
        pw[k] = pk(__ldg(a.W + f0), 2 * p + 1 < NF ? __ldg(a.W + f0 + N) : 0.0f);
      }
    }
  };
  auto store_plane = [&](int slot) {
#pragma unroll
    for (int k = 0; k < kItems; ++k)
      if (islot[k] >= 0) {
        sU[slot * kSPlane * NP + islot[k]] = pu[k];
        sW[slot * kSPlane * NP + islot[k]] = pw[k];
      }
  };

  // element task of this thread
  const int e_raw = tid / G, p_el = tid % G;
  const bool el_ok = e_raw < kSElems && p_el < NP;
  const int e = e_raw < kSElems ? e_raw : kSElems - 1;
  const int pe = p_el < NP ? p_el : NP - 1;
  const int node0 = (e / kSEX) * kSNX + e % kSEX;

  // plane z0 - 1 -> slot 0, then plane z0 in flight
  fetch(z0 - 1);
  store_plane(0);
  fetch(z0);

  for (int i = 0; i <= cz + 1; ++i) {
    // stage plane z0 + i; then gather node plane z0 - 2 + i and compute element
    // layer z0 - 1 + i (between planes z0 - 1 + i and z0 + i) with one barrier:
    // the rings (4 planes, 2 lower-face and 3 upper-face layers) keep what one
    // phase writes apart from what the other reads
    if (i <= cz) {
      store_plane((i + 1) % 4);
      if (i < cz) fetch(z0 + i + 1);
    }
    __syncthreads();

    if (i >= 2) {  // node plane z0 - 2 + i: lower faces of layer i - 1, upper faces of layer i - 2
      const int gz = z0 - 2 + i;
      const u64* sLow = sLowB + ((i - 1) & 1) * 4 * kSElems * NP;
      const u64* upp = sUpB + ((i - 2) % 3) * 4 * kSElems * NP;
      const int s0 = (i - 1) % 4;
      for (int t = tid; t < kSX * kSY * NP; t += kThreads) {
        const int n = t / NP, p = t % NP;
        const int lx = 1 + n % kSX, ly = 1 + n / kSX;
        const int gx = x0 + lx - 1, gy = y0 + ly - 1;
        if (gx >= a.nx || gy >= a.ny) continue;
        u64 acc = sLow[(ly * kSEX + lx) * NP + p];  // corner 0 of the element above
#pragma unroll
        for (int k = 1; k < 8; ++k) {  // element with corner k at this node
          const int ex = lx - (k & 1), ey = ly - ((k >> 1) & 1);
          const u64* src = (k >> 2) ? upp : sLow;
          acc = add2(acc, src[((k & 3) * kSElems + ey * kSEX + ex) * NP + p]);
        }
        // G = (u - u^n)/dt + L (F + kappa K u) / m   or   v/dt + L (H v + kappa K v) / m,
        // the element sums carrying weight |cell|/8 over the interior mass |cell|
        const int c0 = (s0 * kSPlane + ly * kSNX + lx) * NP + p;
        const u64 own = kJVP ? sW[c0] : sub2(sU[c0], sW[c0]);
        u64 r = fma2(own, bc(a.inv_dt), mul2(bc(0.125f * a.mob), acc));
        if (a.unscaled) {
          const float wx = (gx == 0 || gx == a.nx - 1) ? 0.5f : 1.0f;
          const float wy = (gy == 0 || gy == a.ny - 1) ? 0.5f : 1.0f;
          const float wz = (gz == 0 || gz == a.nz - 1) ? 0.5f : 1.0f;
          r = mul2(r, bc(a.cell * wx * wy * wz));
        }
        const int64_t o = (int64_t)gz * plane + (int64_t)gy * a.nx + gx;
        a.out[(int64_t)(2 * p) * N + o] = plo(r);
        if (2 * p + 1 < NF) a.out[(int64_t)(2 * p + 1) * N + o] = phi(r);
      }
    }

    if (i <= cz) {
      const int s0 = i % 4, s1 = (i + 1) % 4;
    {
      // the gradient term acts on v (JVP) or on U (residual)
      u64 c[8], uq[8], vq[8], hq[8], out[8], gx[4], gy[4], gz[4];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        c[k] = sU[(((k >> 2) ? s1 : s0) * kSPlane + node0 + ((k >> 1) & 1) * kSNX + (k & 1)) * NP + pe];
      if constexpr (kJVP) {
        interp3(c, uq);
#pragma unroll
        for (int k = 0; k < 8; ++k)
          c[k] = sW[(((k >> 2) ? s1 : s0) * kSPlane + node0 + ((k >> 1) & 1) * kSNX + (k & 1)) * NP + pe];
        interp3_grad(c, vq, gx, gy, gz);
      } else {
        interp3_grad(c, uq, gx, gy, gz);
      }
      if (a.double_well) {
        // f = W u^2 (1-u)^2:  f' = 2W u (1-u)(1-2u),  f'' = 2W (1 - 6u + 6u^2)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const u64 u = uq[q];
          if constexpr (kJVP) {
            const u64 f2 = fma2(bc(6.0f), sub2(mul2(u, u), u), bc(1.0f));
            hq[q] = mul2(mul2(bc(a.dw2), f2), vq[q]);
          } else {
            const u64 om = sub2(bc(1.0f), u);             // 1 - u
            const u64 o2 = fma2(bc(-2.0f), u, bc(1.0f));  // 1 - 2u
            hq[q] = mul2(mul2(bc(a.dw2), u), mul2(om, o2));
          }
        }
      } else {
        // Fan-Chen: f'_f = u_f (-a + 2g S2 + (b - 2g) u_f^2)
        //           (H v)_f = (-a + 2g S2 + (3b - 6g) u_f^2) v_f + 4g u_f T
        float s2[8], t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const u64 uu = mul2(uq[q], uq[q]);
          s2[q] = p_el < NP ? plo(uu) + phi(uu) : 0.0f;
          if constexpr (kJVP) {
            const u64 uv = mul2(uq[q], vq[q]);
            t[q] = p_el < NP ? plo(uv) + phi(uv) : 0.0f;
          }
        }
        if constexpr (G >= 2) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            s2[q] += __shfl_xor_sync(0xffffffffu, s2[q], 1);
            if constexpr (kJVP) t[q] += __shfl_xor_sync(0xffffffffu, t[q], 1);
          }
        }
        if constexpr (G >= 4) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            s2[q] += __shfl_xor_sync(0xffffffffu, s2[q], 2);
            if constexpr (kJVP) t[q] += __shfl_xor_sync(0xffffffffu, t[q], 2);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const u64 u = uq[q];
          const float base = fmaf(a.two_gamma, s2[q], -a.alpha);
          if constexpr (kJVP)
            hq[q] = fma2(fma2(bc(a.c3b6g), mul2(u, u), bc(base)), vq[q],
                         mul2(bc(a.four_gamma * t[q]), u));
          else
            hq[q] = mul2(u, fma2(bc(a.cb2g), mul2(u, u), bc(base)));
        }
      }
      project3_grad(hq, gx, gy, gz, a.kg, out);
      if (el_ok) {
        u64* sLow = sLowB + (i & 1) * 4 * kSElems * NP;
        u64* up = sUpB + (i % 3) * 4 * kSElems * NP;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          sLow[(k * kSElems + e) * NP + p_el] = out[k];
          up[(k * kSElems + e) * NP + p_el] = out[4 + k];
        }
      }
    }
    }
  }
  }  // segments
}

template <int NF, bool kJVP>
cudaError_t launch_sweep_nf(const Implicit3DArgs& a, cudaStream_t s) {
  constexpr int NP = (NF + 1) / 2;
  constexpr size_t smem = SweepCfg<NP>::kSmem;
  static std::atomic<unsigned long long> raised{0};
  const cudaError_t e = raise_smem_limit(k_implicit3d_sweep<NF, kJVP>, (int)smem, raised);
  if (e != cudaSuccess) return e;
  // one wave of resident blocks, each sweeping an equal share of the column
  // planes (no more blocks than column planes)
  static std::atomic<int> per_sm{0};
  if (per_sm.load() == 0) {
    int n = 0;
    const cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, k_implicit3d_sweep<NF, kJVP>, SweepCfg<NP>::kThreads, smem);
    if (oe != cudaSuccess) return oe;
    per_sm.store(n > 0 ? n : 1);
  }
  const int64_t planes = (int64_t)((a.nx + kSX - 1) / kSX) * ((a.ny + kSY - 1) / kSY) * a.nz;
  const int64_t blocks = std::min<int64_t>(planes, (int64_t)per_sm.load() * device_sm_count());
  k_implicit3d_sweep<NF, kJVP><<<(unsigned)blocks, SweepCfg<NP>::kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool kJVP>
cudaError_t launch_sweep_any(const Implicit3DArgs& a, cudaStream_t s) {
  switch (a.nf) {
    case 1: return launch_sweep_nf<1, kJVP>(a, s);
    case 2: return launch_sweep_nf<2, kJVP>(a, s);
    case 3: return launch_sweep_nf<3, kJVP>(a, s);
    case 4: return launch_sweep_nf<4, kJVP>(a, s);
    case 5: return launch_sweep_nf<5, kJVP>(a, s);
    case 6: return launch_sweep_nf<6, kJVP>(a, s);
    case 7: return launch_sweep_nf<7, kJVP>(a, s);
    case 8: return launch_sweep_nf<8, kJVP>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_residual3d(const Implicit3DArgs& a, cudaStream_t s) {
  return launch_sweep_any<false>(a, s);
}

cudaError_t launch_jvp3d(const Implicit3DArgs& a, cudaStream_t s) { return launch_sweep_any<true>(a, s); }

}  // namespace pf
