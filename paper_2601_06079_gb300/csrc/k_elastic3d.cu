// Eshelby-inclusion elasticity on a 3-D Q1 grid (JAX-PF Eq. 3-4, eigenstrain
// of Supp. 3 Eq. III.1): the matrix-free stiffness K u of small-strain
// isotropic elasticity, the eigenstrain load f = int B^T C eps0, and the two
// fused conjugate-gradient updates.  Displacements are component-major FP32
// planes u[c * N + node], c = x, y, z.
//
// K u is node-centric and needs no atomics: a thread sweeps a column of nodes
// along z with the 3 x 3 x 3 neighbourhood of all three components in
// registers (one new 3 x 3 plane, 27 loads coalesced along x, per node) and
// applies
//   interior nodes: the assembled 27-point stencil, 3 x 3 coefficients per
//                   offset (243 FMA);
//   boundary nodes: the element stiffness of each of its (up to 8) elements
//                   that lie inside the mesh, row block of the node's corner.
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

// FP64 sum over the block (any block shape up to 1024 threads), result in thread 0
__device__ double block_sum(double v) {
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

constexpr int kBX = 32, kBY = 4;  // (x, y) columns per block
constexpr int kZChunk = 16;        // nodes per column and thread

// load the 3 x 3 (x, y) neighbourhood of plane z (clamped into the mesh)
__device__ __forceinline__ void load_plane(const Elastic3DArgs& a, int64_t N, int x, int y, int z,
                                           float p[9][3]) {
  const int zz = clampi(z, 0, a.nz - 1);
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    const int yy = clampi(y + dy, 0, a.ny - 1);
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int xx = clampi(x + dx, 0, a.nx - 1);
      const int64_t g = ((int64_t)zz * a.ny + yy) * a.nx + xx;
#pragma unroll
      for (int c = 0; c < 3; ++c) p[(dy + 1) * 3 + (dx + 1)][c] = __ldg(a.u + c * N + g);
    }
  }
}

// One thread per (x, y) column and chunk of kZChunk nodes along z: a window
// of three planes of the 3 x 3 neighbourhood slides down z in registers, so
// each node costs one plane of 27 loads instead of its 81 neighbours.
//
// With a.dot set, each block also writes the FP64 partial sum of u . Ku over
// its nodes to a.dot[block] (fixed order: the CG step's p . Ap).
template <bool kDot>
__global__ void __launch_bounds__(kBX * kBY) k_elastic_apply(const Elastic3DArgs a) {
  const int64_t N = (int64_t)a.nx * a.ny * a.nz;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  float dot = 0.0f;  // this thread's at most kZChunk nodes; blocks sum in FP64
  if (x < a.nx && y < a.ny) {
  const int z0 = blockIdx.z * kZChunk, z1 = min(z0 + kZChunk, a.nz);
  float pm[9][3], pc[9][3], pp[9][3];  // planes z - 1, z, z + 1 (rows beyond the mesh clamped)
  load_plane(a, N, x, y, z0 - 1, pm);
  load_plane(a, N, x, y, z0, pc);
  const bool xy_in = x > 0 && y > 0 && x < a.nx - 1 && y < a.ny - 1;
  for (int z = z0; z < z1; ++z) {
    load_plane(a, N, x, y, z + 1, pp);
    // neighbourhood o = (dz+1)*9 + (dy+1)*3 + (dx+1) as differences to the
    // node's own values (o = 13 is the node itself)
    float v[27][3];
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v[k][c] = pm[k][c] - pc[4][c];
        v[9 + k][c] = pc[k][c] - pc[4][c];
        v[18 + k][c] = pp[k][c] - pc[4][c];
      }
    float out[3] = {0.0f, 0.0f, 0.0f};
    if (xy_in && z > 0 && z < a.nz - 1) {
#pragma unroll
      for (int o = 0; o < 27; ++o)
        if (o != 13) {
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) out[i] = fmaf(a.ks[(o * 3 + i) * 3 + j], v[o][j], out[i]);
        }
    } else {
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
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
              out[i] = fmaf(a.ke[(oct * 3 + i) * 24 + b * 3 + j], v[o][j], out[i]);
        }
      }
    }
    if (a.constrain) {  // symmetry planes: u_x on x = 0, u_y on y = 0, u_z on z = 0
      if (x == 0) out[0] = 0.0f;
      if (y == 0) out[1] = 0.0f;
      if (z == 0) out[2] = 0.0f;
    }
    const int64_t node = ((int64_t)z * a.ny + y) * a.nx + x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a.out[c * N + node] = out[c];
      if (kDot) dot = fmaf(pc[4][c], out[c], dot);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pm[k][c] = pc[k][c];
        pc[k][c] = pp[k][c];
      }
  }
  }
  if (kDot) {
    const double s = block_sum((double)dot);
    if (threadIdx.x == 0 && threadIdx.y == 0)
      a.dot[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
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
__global__ void k_cg_xr(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
                        const float* __restrict__ Ap, int64_t n, const double* __restrict__ sc,
                        int slot, double* __restrict__ part) {
  const float alpha = (float)(sc[slot] / sc[2]);
  double rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fmaf(alpha, p[i], x[i]);
    const float ri = fmaf(-alpha, Ap[i], r[i]);
    r[i] = ri;
    rr += (double)(ri * ri);
  }
  const double s = block_sum(rr);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out = sum of part[0 .. nb) in a fixed order (one block)
__global__ void k_sum_part(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
  const double s = block_sum(v);
  if (threadIdx.x == 0) *out = s;
}

//   p = r + beta p   with beta = sc[1 - slot] / sc[slot]
__global__ void k_cg_p(const float* __restrict__ r, float* __restrict__ p, int64_t n,
                       const double* __restrict__ sc, int slot) {
  const float beta = (float)(sc[1 - slot] / sc[slot]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fmaf(beta, p[i], r[i]);
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
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 8 ? b : 152 * 8);
}

}  // namespace

int elastic_apply_blocks(int nx, int ny, int nz) {
  return ((nx + kBX - 1) / kBX) * ((ny + kBY - 1) / kBY) * ((nz + kZChunk - 1) / kZChunk);
}

int cg_blocks() { return 152 * 8; }

cudaError_t launch_elastic_apply(const Elastic3DArgs& a, cudaStream_t s) {
  const dim3 grid((a.nx + kBX - 1) / kBX, (a.ny + kBY - 1) / kBY, (a.nz + kZChunk - 1) / kZChunk);
  if (a.dot)
    k_elastic_apply<true><<<grid, dim3(kBX, kBY), 0, s>>>(a);
  else
    k_elastic_apply<false><<<grid, dim3(kBX, kBY), 0, s>>>(a);
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
  k_cg_xr<<<cg_blocks(), 256, 0, s>>>(x, r, p, Ap, n, sc, slot, part);
  return cudaGetLastError();
}

cudaError_t launch_cg_p(const float* r, float* p, int64_t n, const double* sc, int slot,
                        cudaStream_t s) {
  k_cg_p<<<blocks_for(n), 256, 0, s>>>(r, p, n, sc, slot);
  return cudaGetLastError();
}

}  // namespace pf
