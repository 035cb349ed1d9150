// Eshelby-inclusion elasticity on a 3-D Q1 grid (JAX-PF Eq. 3-4, eigenstrain
// of Supp. 3 Eq. III.1): the matrix-free stiffness K u of small-strain
// isotropic elasticity, the eigenstrain load f = int B^T C eps0, and the two
// fused conjugate-gradient updates.  Displacements are component-major FP32
// planes u[c * N + node], c = x, y, z.
//
// K u is node-centric and needs no atomics, in two launches:
//   interior nodes: a thread sweeps a column along z with the 3 x 3 x 3
//                   neighbourhood of all three components in registers (one
//                   new plane, 27 loads coalesced along x, per node) and
//                   applies the assembled 27-point stencil, 3 x 3
//                   coefficients per offset;
//   boundary nodes: one thread per node applies the element stiffness of
//                   each of its (up to 8) elements that lie inside the mesh,
//                   row block of the node's corner.
// Both coefficient tables come from the element stiffness of the uniform
// box element in closed form (host, FP64) and travel as kernel parameters,
// whose uniform reads feed the FMAs directly.  K annihilates translations, so
// both act on differences u(neighbour) - u(node): for smooth fields the sum
// of 27 products cancels by about n^2, and the differences keep that
// cancellation out of FP32 (the centre coefficient drops out).
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kThreads = 128;

// Sum over the block (any block shape up to 1024 threads), result in thread
// 0: warp sums in FP32 (GB300 issues about 2 FP64 operations per clock per
// SM, 64 times fewer than FP32), the warp partials in FP64, fixed order
__device__ double block_sum(float v) {
  __shared__ double part[32];
  const int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((t & 31) == 0) part[t >> 5] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (t == 0)
    for (int w = 0; w < (nt + 31) / 32; ++w) s += part[w];
  return s;
}

// the same for FP64 inputs (the single-block sum of the block partials)
__device__ double block_sum_f64(double v) {
  __shared__ double part[32];
  const int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((t & 31) == 0) part[t >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (t == 0)
    for (int w = 0; w < (nt + 31) / 32; ++w) s += part[w];
  return s;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

constexpr int kBX = 32, kBY = 4;  // (x, y) columns per interior block (kBX * kBY = kThreads)
constexpr int kZChunk = 15;        // interior nodes per column and thread (a multiple of 3)

// 3 x 3 (x, y) neighbourhood of interior column (x, y) in plane z
__device__ __forceinline__ void load_plane(const float* __restrict__ u, int64_t N, int64_t nx,
                                           int64_t row0, float p[9][3]) {
  // row0: index of node (x - 1, y - 1) in plane z
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
      for (int c = 0; c < 3; ++c) p[dy * 3 + dx][c] = __ldg(u + c * N + row0 + dy * nx + dx);
}

// K u at an interior node from its three planes, on differences to the node.
// The assembled stencil of the uniform isotropic grid is centrally symmetric,
// K(-o) = K(o), so each mirror pair of offsets acts once on the sum of its two
// differences; and a coupling K_ij(o), i != j, is a product of central
// differences along i and j, so it vanishes unless o_i and o_j are both
// nonzero -- those terms are left out at compile time (75 FMA instead of 234).
__device__ __forceinline__ void interior_node(const Elastic3DArgs& a, const float (&pm)[9][3],
                                              const float (&pc)[9][3], const float (&pp)[9][3],
                                              float out[3]) {
  out[0] = out[1] = out[2] = 0.0f;
#pragma unroll
  for (int o = 14; o < 27; ++o) {  // one offset of each pair (o, 26 - o)
    const int m = 26 - o;
    const int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
    const float(&po)[9][3] = o < 9 ? pm : (o < 18 ? pc : pp);
    const float(&pq)[9][3] = m < 9 ? pm : (m < 18 ? pc : pp);
    float s[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) s[j] = (po[o % 9][j] - pc[4][j]) + (pq[m % 9][j] - pc[4][j]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      out[i] = fmaf(a.ks[(o * 3 + i) * 3 + i], s[i], out[i]);
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (j != i && off[i] != 0 && off[j] != 0)
          out[i] = fmaf(a.ks[(o * 3 + i) * 3 + j], s[j], out[i]);
    }
  }
}

// Interior nodes (1 <= x, y, z <= n - 2): one thread per (x, y) column and
// kZChunk nodes along z.  Three planes of the 3 x 3 neighbourhood rotate
// through registers (the loop is unrolled by 3, so the rotation is renaming),
// and each node costs one plane of 27 loads at unclamped row addresses.
// With kDot each block writes the FP64 partial of u . Ku over its nodes to
// a.dot[block] (fixed order).
#ifndef PF_EL_MINB
#define PF_EL_MINB 4  // minimum resident interior blocks per SM asked of the register allocator
#endif
#ifndef PF_EL_UNROLL3
#define PF_EL_UNROLL3 0  // 1: z loop unrolled by 3 (plane rotation by renaming, more registers)
#endif

template <bool kDot>
__device__ __forceinline__ float interior_block(const Elastic3DArgs& a, int bx, int by, int bz) {
  const int64_t N = (int64_t)a.nx * a.ny * a.nz;
  const int64_t nx = a.nx, plane = (int64_t)a.nx * a.ny;
  const int x = 1 + bx * kBX + (threadIdx.x % kBX), y = 1 + by * kBY + (threadIdx.x / kBX);
  float dot = 0.0f;  // this thread's at most kZChunk nodes; blocks sum in FP64
  if (x < a.nx - 1 && y < a.ny - 1) {
    const int z0 = 1 + bz * kZChunk, z1 = min(z0 + kZChunk, a.nz - 1);
    const int64_t col0 = (int64_t)(y - 1) * nx + (x - 1);
    float P0[9][3], P1[9][3], P2[9][3];
    load_plane(a.u, N, nx, (z0 - 1) * plane + col0, P0);
    load_plane(a.u, N, nx, z0 * plane + col0, P1);
    auto node = [&](int z, const float(&pm)[9][3], const float(&pc)[9][3],
                    const float(&pp)[9][3]) {
      float out[3];
      interior_node(a, pm, pc, pp, out);
      const int64_t g = z * plane + col0 + nx + 1;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a.out[c * N + g] = out[c];
        if (kDot) dot = fmaf(pc[4][c], out[c], dot);
      }
    };
#if PF_EL_UNROLL3
    for (int z = z0; z < z1; z += 3) {
      load_plane(a.u, N, nx, (z + 1) * plane + col0, P2);
      node(z, P0, P1, P2);
      if (z + 1 >= z1) break;
      load_plane(a.u, N, nx, (z + 2) * plane + col0, P0);
      node(z + 1, P1, P2, P0);
      if (z + 2 >= z1) break;
      load_plane(a.u, N, nx, (z + 3) * plane + col0, P1);
      node(z + 2, P2, P0, P1);
    }
#else
#pragma unroll 1
    for (int z = z0; z < z1; ++z) {
      load_plane(a.u, N, nx, (z + 1) * plane + col0, P2);
      node(z, P0, P1, P2);
#pragma unroll
      for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          P0[k][c] = P1[k][c];
          P1[k][c] = P2[k][c];
        }
    }
#endif
  }
  return dot;
}

// boundary node number i -> (x, y, z): the two z faces, then the two y faces
// without their z rows, then the two x faces without their y and z rows
__device__ __forceinline__ void boundary_node(int64_t i, int nx, int ny, int nz, int& x, int& y,
                                              int& z) {
  const int64_t fz = (int64_t)nx * ny, fy = (int64_t)nx * (nz - 2);
  if (i < 2 * fz) {
    z = i < fz ? 0 : nz - 1;
    const int64_t r = i % fz;
    y = (int)(r / nx);
    x = (int)(r % nx);
  } else if ((i -= 2 * fz) < 2 * fy) {
    y = i < fy ? 0 : ny - 1;
    const int64_t r = i % fy;
    z = 1 + (int)(r / nx);
    x = (int)(r % nx);
  } else {
    i -= 2 * fy;
    const int64_t fx = (int64_t)(ny - 2) * (nz - 2);
    x = i < fx ? 0 : nx - 1;
    const int64_t r = i % fx;
    z = 1 + (int)(r / (ny - 2));
    y = 1 + (int)(r % (ny - 2));
  }
}

__host__ __device__ int64_t boundary_count(int nx, int ny, int nz) {
  return 2 * (int64_t)nx * ny + 2 * (int64_t)nx * (nz - 2) + 2 * (int64_t)(ny - 2) * (nz - 2);
}

// Boundary nodes: one thread per node, its 3 x 3 x 3 neighbourhood (clamped
// into the mesh) as differences, and the element-stiffness row blocks of the
// (up to 8) elements inside the mesh; then the symmetry-plane constraints.
template <bool kDot>
__device__ __forceinline__ float boundary_block(const Elastic3DArgs& a, int blk) {
  const int64_t N = (int64_t)a.nx * a.ny * a.nz;
  const int64_t nb = boundary_count(a.nx, a.ny, a.nz);
  const int64_t i = (int64_t)blk * kThreads + threadIdx.x;
  float dot = 0.0f;
  if (i < nb) {
    int x, y, z;
    boundary_node(i, a.nx, a.ny, a.nz, x, y, z);
    float v[27][3];
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = clampi(z + dz, 0, a.nz - 1);
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = clampi(y + dy, 0, a.ny - 1);
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = clampi(x + dx, 0, a.nx - 1);
          const int64_t g = ((int64_t)zz * a.ny + yy) * a.nx + xx;
#pragma unroll
          for (int c = 0; c < 3; ++c) v[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)][c] = __ldg(a.u + c * N + g);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < 27; ++o)
      if (o != 13) {
#pragma unroll
        for (int c = 0; c < 3; ++c) v[o][c] -= v[13][c];
      }
    float out[3] = {0.0f, 0.0f, 0.0f};
    // element with lower corner (x - ox, y - oy, z - oz): this node is its
    // corner a = ox + 2 oy + 4 oz; its corner b is at offset (b - a) per axis
#pragma unroll
    for (int oct = 0; oct < 8; ++oct) {
      const int ox = oct & 1, oy = (oct >> 1) & 1, oz = oct >> 2;
      const int ex = x - ox, ey = y - oy, ez = z - oz;
      if (ex < 0 || ey < 0 || ez < 0 || ex > a.nx - 2 || ey > a.ny - 2 || ez > a.nz - 2) continue;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
        const int o = (bz - oz + 1) * 9 + (by - oy + 1) * 3 + (bx - ox + 1);
        if (o == 13) continue;  // the node itself: a zero difference
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            out[ii] = fmaf(a.ke[(oct * 3 + ii) * 24 + b * 3 + j], v[o][j], out[ii]);
      }
    }
    if (a.constrain) {  // symmetry planes: u_x on x = 0, u_y on y = 0, u_z on z = 0
      if (x == 0) out[0] = 0.0f;
      if (y == 0) out[1] = 0.0f;
      if (z == 0) out[2] = 0.0f;
    }
    const int64_t g = ((int64_t)z * a.ny + y) * a.nx + x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a.out[c * N + g] = out[c];
      if (kDot) dot = fmaf(v[13][c], out[c], dot);
    }
  }
  return dot;
}

// One launch for both: blocks [0, ni) are interior column blocks (gx x gy x gz
// of them), the rest boundary blocks, so the boundary work fills the tail of
// the interior wave.  With kDot each block writes the FP64 partial of u . Ku
// over its nodes to a.dot[block] (fixed order).
template <bool kDot>
__global__ void __launch_bounds__(kThreads, PF_EL_MINB) k_elastic_apply(const Elastic3DArgs a, int gx,
                                                                       int gy, int ni) {
  const int b = blockIdx.x;
  float dot;
  if (b < ni)
    dot = interior_block<kDot>(a, b % gx, (b / gx) % gy, b / (gx * gy));
  else
    dot = boundary_block<kDot>(a, b - ni);
  if (kDot) {
    const double s = block_sum(dot);
    if (threadIdx.x == 0) a.dot[b] = s;
  }
}

// f_i(node) = sum over its elements and their Gauss points of
// w d_i N_a(q) s(q), s = scale * (1 - tanh(l (|x_q| - a))) / 2  (eigenstrain
// load with scale = (3 lam + 2 mu) m), or s = scale (unit: the volume functional)
__global__ void __launch_bounds__(kThreads) k_elastic_load(ElasticLoadArgs a, float* f) {
  const int64_t N = (int64_t)a.nx * a.ny * a.nz;
  const int64_t node = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (node >= N) return;
  const int x = (int)(node % a.nx), y = (int)((node / a.nx) % a.ny), z = (int)(node / ((int64_t)a.nx * a.ny));
  const float g[2] = {0.5f - 0.28867513459481287f, 0.5f + 0.28867513459481287f};
  float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int oct = 0; oct < 8; ++oct) {
    const int ox = oct & 1, oy = (oct >> 1) & 1, oz = oct >> 2;
    const int ex = x - ox, ey = y - oy, ez = z - oz;
    if (ex < 0 || ey < 0 || ez < 0 || ex > a.nx - 2 || ey > a.ny - 2 || ez > a.nz - 2) continue;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float s = g[q & 1], t = g[(q >> 1) & 1], w = g[q >> 2];
      float sv = a.scale;
      if (!a.unit) {
        const float px = (ex + s) * a.hx, py = (ey + t) * a.hy, pz = (ez + w) * a.hz;
        const float r = sqrtf(px * px + py * py + pz * pz);
        sv *= 0.5f * (1.0f - tanhf(a.l * (r - a.a)));
      }
      // shape function of corner (ox, oy, oz) and its gradient at (s, t, w)
      const float nx_ = ox ? s : 1.0f - s, ny_ = oy ? t : 1.0f - t, nz_ = oz ? w : 1.0f - w;
      const float sx = ox ? 1.0f : -1.0f, sy = oy ? 1.0f : -1.0f, sz = oz ? 1.0f : -1.0f;
      const float wq = a.wq * sv;
      acc[0] = fmaf(wq, sx * a.ihx * ny_ * nz_, acc[0]);
      acc[1] = fmaf(wq, nx_ * sy * a.ihy * nz_, acc[1]);
      acc[2] = fmaf(wq, nx_ * ny_ * sz * a.ihz, acc[2]);
    }
  }
  if (a.constrain) {
    if (x == 0) acc[0] = 0.0f;
    if (y == 0) acc[1] = 0.0f;
    if (z == 0) acc[2] = 0.0f;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) f[c * N + node] = acc[c];
}

// CG, with the scalars on the device: sc[0], sc[1] = r.r (ping-pong by
// iteration parity `slot`), sc[2] = p.Ap.
//   x += alpha p, r -= alpha Ap   with alpha = sc[slot] / sc[2]
//   and part[block] = the block's FP64 partial of the new r . r
//   (float4 over the first 4 n4 entries -- n4 = 0 unless every vector is
//   16-byte aligned -- and scalars over the rest)
__global__ void k_cg_xr(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
                        const float* __restrict__ Ap, int64_t n, int64_t n4,
                        const double* __restrict__ sc, int slot, double* __restrict__ part) {
  const float alpha = (float)(sc[slot] / sc[2]);
  float rr = 0.0f;  // at most a few dozen squares per thread; blocks sum in FP64
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n4; i += nth) {
    float4 xv = reinterpret_cast<float4*>(x)[i], rv = reinterpret_cast<float4*>(r)[i];
    const float4 pv = reinterpret_cast<const float4*>(p)[i], av = reinterpret_cast<const float4*>(Ap)[i];
    xv.x = fmaf(alpha, pv.x, xv.x);
    xv.y = fmaf(alpha, pv.y, xv.y);
    xv.z = fmaf(alpha, pv.z, xv.z);
    xv.w = fmaf(alpha, pv.w, xv.w);
    rv.x = fmaf(-alpha, av.x, rv.x);
    rv.y = fmaf(-alpha, av.y, rv.y);
    rv.z = fmaf(-alpha, av.z, rv.z);
    rv.w = fmaf(-alpha, av.w, rv.w);
    reinterpret_cast<float4*>(x)[i] = xv;
    reinterpret_cast<float4*>(r)[i] = rv;
    rr = fmaf(rv.x, rv.x, rr);
    rr = fmaf(rv.y, rv.y, rr);
    rr = fmaf(rv.z, rv.z, rr);
    rr = fmaf(rv.w, rv.w, rr);
  }
  for (int64_t i = 4 * n4 + tid; i < n; i += nth) {
    x[i] = fmaf(alpha, p[i], x[i]);
    const float ri = fmaf(-alpha, Ap[i], r[i]);
    r[i] = ri;
    rr = fmaf(ri, ri, rr);
  }
  const double s = block_sum(rr);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out = sum of part[0 .. nb) in a fixed order (one block)
__global__ void k_sum_part(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
  const double s = block_sum_f64(v);
  if (threadIdx.x == 0) *out = s;
}

//   p = r + beta p   with beta = sc[1 - slot] / sc[slot]
__global__ void k_cg_p(const float* __restrict__ r, float* __restrict__ p, int64_t n, int64_t n4,
                       const double* __restrict__ sc, int slot) {
  const float beta = (float)(sc[1 - slot] / sc[slot]);
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n4; i += nth) {
    float4 pv = reinterpret_cast<float4*>(p)[i];
    const float4 rv = reinterpret_cast<const float4*>(r)[i];
    pv.x = fmaf(beta, pv.x, rv.x);
    pv.y = fmaf(beta, pv.y, rv.y);
    pv.z = fmaf(beta, pv.z, rv.z);
    pv.w = fmaf(beta, pv.w, rv.w);
    reinterpret_cast<float4*>(p)[i] = pv;
  }
  for (int64_t i = 4 * n4 + tid; i < n; i += nth) p[i] = fmaf(beta, p[i], r[i]);
}

// zero the constrained entries (symmetry planes) of a displacement vector
__global__ void k_elastic_constrain(float* __restrict__ v, int nx, int ny, int nz) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < N;
       node += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(node % nx), y = (int)((node / nx) % ny), z = (int)(node / ((int64_t)nx * ny));
    if (x == 0) v[node] = 0.0f;
    if (y == 0) v[N + node] = 0.0f;
    if (z == 0) v[2 * N + node] = 0.0f;
  }
}

int blocks_for(int64_t n) {
  const int64_t b = (n + 255) / 256, cap = 8 * (int64_t)device_sm_count();
  return (int)(b < cap ? b : cap);
}

dim3 interior_grid(int nx, int ny, int nz) {
  if (nx < 3 || ny < 3 || nz < 3) return dim3(0, 0, 0);
  return dim3((nx - 2 + kBX - 1) / kBX, (ny - 2 + kBY - 1) / kBY, (nz - 2 + kZChunk - 1) / kZChunk);
}

int boundary_blocks(int nx, int ny, int nz) {
  return (int)((boundary_count(nx, ny, nz) + kThreads - 1) / kThreads);
}

}  // namespace

int elastic_apply_blocks(int nx, int ny, int nz) {
  const dim3 g = interior_grid(nx, ny, nz);
  return (int)(g.x * g.y * g.z) + boundary_blocks(nx, ny, nz);
}

// 8 blocks per SM, fixed per device (the r.r partials are summed in a fixed order)
int cg_blocks() { return 8 * device_sm_count(); }

cudaError_t launch_elastic_apply(const Elastic3DArgs& a, cudaStream_t s) {
  const dim3 gi = interior_grid(a.nx, a.ny, a.nz);
  const int ni = (int)(gi.x * gi.y * gi.z), nb = boundary_blocks(a.nx, a.ny, a.nz);
  if (a.dot)
    k_elastic_apply<true><<<ni + nb, kThreads, 0, s>>>(a, (int)gi.x, (int)gi.y, ni);
  else
    k_elastic_apply<false><<<ni + nb, kThreads, 0, s>>>(a, (int)gi.x, (int)gi.y, ni);
  return cudaGetLastError();
}

cudaError_t launch_sum_part(const double* part, int nb, double* out, cudaStream_t s) {
  k_sum_part<<<1, 256, 0, s>>>(part, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_elastic_load(const ElasticLoadArgs& a, float* f, cudaStream_t s) {
  const int64_t N = (int64_t)a.nx * a.ny * a.nz;
  k_elastic_load<<<(unsigned)((N + kThreads - 1) / kThreads), kThreads, 0, s>>>(a, f);
  return cudaGetLastError();
}

cudaError_t launch_elastic_constrain(float* v, int nx, int ny, int nz, cudaStream_t s) {
  k_elastic_constrain<<<blocks_for((int64_t)nx * ny * nz), 256, 0, s>>>(v, nx, ny, nz);
  return cudaGetLastError();
}

cudaError_t launch_cg_xr(float* x, float* r, const float* p, const float* Ap, int64_t n,
                         const double* sc, int slot, double* part, cudaStream_t s) {
  const bool al = (((uintptr_t)x | (uintptr_t)r | (uintptr_t)p | (uintptr_t)Ap) & 15) == 0;
  k_cg_xr<<<cg_blocks(), 256, 0, s>>>(x, r, p, Ap, n, al ? n / 4 : 0, sc, slot, part);
  return cudaGetLastError();
}

cudaError_t launch_cg_p(const float* r, float* p, int64_t n, const double* sc, int slot,
                        cudaStream_t s) {
  const bool al = (((uintptr_t)r | (uintptr_t)p) & 15) == 0;
  k_cg_p<<<blocks_for(n), 256, 0, s>>>(r, p, n, al ? n / 4 : 0, sc, slot);
  return cudaGetLastError();
}

}  // namespace pf
