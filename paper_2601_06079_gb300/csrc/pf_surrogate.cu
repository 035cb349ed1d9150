// Learned warm start for the implicit step: a small 3-D U-Net (4 levels, 32
// channels, 3x3x3 convolutions, BF16 operands with FP32 accumulation) that
// maps U^n (and up to two earlier states) to a correction of the first Newton
// iterate for U^{n+1}.  Forward, backward and the Adam update all run in this
// library's kernels; the caller owns every buffer.
//
// Layers (input channels padded 8/16/24 -> 32, output 16 -> first 8 used):
//   level 0: c0 32->32, c1 32->32 (skip s0) ; pool
//   level 1: c2, c3 (skip s1) ; pool      level 2: c4, c5 (skip s2) ; pool
//   level 3: c6, c7 ; up + s2 -> c8, c9 ; up + s1 -> c10, c11 ; up + s0 -> c12, c13
//   c14 32->16 (no ReLU) -> increment.
// Parameters: FP32 master copy, per layer [27][c_out][c_in] weights then c_out
// biases; BF16 copies (forward and tap-reversed transposed for the data
// gradient) are derived every call.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pf_internal.h"

namespace {

struct LayerDef {
  int cin, cout, relu, level;
};

constexpr int kNL = 15;
constexpr LayerDef kLayers[kNL] = {
    {32, 32, 1, 0}, {32, 32, 1, 0}, {32, 32, 1, 1}, {32, 32, 1, 1}, {32, 32, 1, 2},
    {32, 32, 1, 2}, {32, 32, 1, 3}, {32, 32, 1, 3}, {32, 32, 1, 2}, {32, 32, 1, 2},
    {32, 32, 1, 1}, {32, 32, 1, 1}, {32, 32, 1, 0}, {32, 32, 1, 0}, {32, 16, 0, 0}};
constexpr int kNF = 8;        // order parameters
constexpr int kC = 32;        // feature channels
constexpr int kCin0 = 32;     // padded input channels
constexpr int kCout = 16;     // padded output channels
// grid of the mma.sync convolution and blocks (partial sums) of the weight
// gradient, per device
int conv_grid() { return 2 * pf::device_sm_count(); }
int wgrad_blocks() { return pf::device_sm_count(); }
// floats of weight-gradient partials: the tcgen05 kernel's or the mma.sync one's
size_t part_floats(int cin, int cout) {
  const size_t a = pf::wgrad_tc_part_floats(), b = (size_t)wgrad_blocks() * 27 * cin * cout;
  return a > b ? a : b;
}
constexpr int kSigBlocks = 256;  // blocks per sample of the increment-scale reduction

int64_t w_count(int l) { return (int64_t)27 * kLayers[l].cin * kLayers[l].cout; }
int64_t w_off(int l) {
  int64_t o = 0;
  for (int i = 0; i < l; ++i) o += w_count(i) + kLayers[i].cout;
  return o;
}
int64_t b_off(int l) { return w_off(l) + w_count(l); }
int64_t param_count() { return w_off(kNL); }

size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct Plan {
  int B, D, H, W;
  int64_t V[4];  // voxels (all samples) per level
  // byte offsets into the workspace
  size_t x16, act[kNL], pool[4], up[4], y32, wf[kNL], wb[kNL];
  size_t gy, g[4][3], grad, part, msep, loss, err, sig, sigo, sigp, res, resq;
  size_t total;
};

Plan make_plan(int B, int D, int H, int W, bool training) {
  Plan p{};
  p.B = B;
  p.D = D;
  p.H = H;
  p.W = W;
  for (int l = 0; l < 4; ++l) p.V[l] = (int64_t)B * (D >> l) * (H >> l) * (W >> l);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += al(bytes);
    return o;
  };
  p.x16 = take(2 * p.V[0] * kCin0);
  for (int l = 0; l < kNL - 1; ++l) p.act[l] = take(2 * p.V[kLayers[l].level] * kC);
  for (int l = 1; l < 4; ++l) {
    p.pool[l] = take(2 * p.V[l] * kC);
    p.up[l - 1] = take(2 * p.V[l - 1] * kC);
  }
  p.y32 = take(4 * p.V[0] * kCout);
  p.err = take(sizeof(int));
  p.sig = take(sizeof(float) * B);
  p.sigo = take(sizeof(float) * B);
  p.sigp = take(sizeof(double) * kSigBlocks * B);
  for (int l = 0; l < kNL; ++l) {
    p.wf[l] = take(2 * w_count(l));
    p.wb[l] = take(2 * w_count(l));
  }
  if (training) {
    p.gy = take(2 * p.V[0] * kCout);
    for (int l = 0; l < 4; ++l)
      for (int k = 0; k < 3; ++k) p.g[l][k] = take(2 * p.V[l] * kC);
    p.grad = take(4 * param_count());
    p.part = take(4 * part_floats(kC, kC));
    p.msep = take(8 * 1024);
    p.res = take(4 * p.V[0] * kNF);
    p.resq = take(4 * p.V[0] * kNF);
    p.loss = take(8);
  }
  p.total = off;
  return p;
}

bool scale_ok(float a) { return a > 0.0f && isfinite(a); }

bool dims_ok(int B, int D, int H, int W) {
  return B >= 1 && D >= 16 && H >= 64 && W >= 64 && D % 16 == 0 && H % 64 == 0 && W % 64 == 0 &&
         (int64_t)B * D * H * W <= ((int64_t)1 << 31);
}

#define SG_CUDA(call)                              \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return PF_ERR_CUDA;     \
  } while (0)

struct Net {
  const Plan& p;
  char* ws;
  cudaStream_t s;
  bool tc;  // tcgen05 convolutions where the level's shape allows
  template <class T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(ws + off);
  }
  int dim(int level, int axis) const { return (axis == 0 ? p.D : axis == 1 ? p.H : p.W) >> level; }
};

pf_status convert_all(const Net& n, const float* params, bool with_bwd) {
  static_assert(kNL <= pf::kMaxConvertLayers, "layer table too small");
  pf::ConvertTable t{};
  for (int l = 0; l < kNL; ++l) {
    t.w[l] = params + w_off(l);
    t.fwd[l] = n.at<void>(n.p.wf[l]);
    t.bwd[l] = with_bwd ? n.at<void>(n.p.wb[l]) : nullptr;
    t.ci[l] = kLayers[l].cin;
    t.co[l] = kLayers[l].cout;
  }
  t.n = kNL;
  SG_CUDA(pf::launch_convert_weights_all(t, n.s));
  return PF_OK;
}

// One convolution: the tcgen05 kernel where the shape allows, else mma.sync.
cudaError_t conv(const Net& n, int cin, int cout, const void* x, const void* wt, const float* bias,
                 int relu, void* y16, float* y32, int d, int h, int w) {
  if (n.tc && pf::conv3d_tc_shape_ok(n.p.B, d, h, w))
    return pf::launch_conv3d_tc(cin, cout, x, wt, bias, relu, y16, y32, n.p.B, d, h, w,
                                n.at<int>(n.p.err), n.s);
  return pf::launch_conv3d(cin, cout, x, wt, bias, relu, y16, y32, n.p.B, d, h, w, conv_grid(),
                           n.s);
}

// Zero the pipeline-timeout flag before a call; read it after the stream
// has been synchronised.
pf_status clear_err(const Net& n) {
  SG_CUDA(cudaMemsetAsync(n.at<int>(n.p.err), 0, sizeof(int), n.s));
  return PF_OK;
}

pf_status check_err(const Net& n) {
  int e = 0;
  SG_CUDA(cudaMemcpyAsync(&e, n.at<int>(n.p.err), sizeof(int), cudaMemcpyDeviceToHost, n.s));
  SG_CUDA(cudaStreamSynchronize(n.s));
  return e ? PF_ERR_TIMEOUT : PF_OK;
}

const void* layer_input(const Net& n, int l) {
  switch (l) {
    case 0: return n.at<void>(n.p.x16);
    case 2: return n.at<void>(n.p.pool[1]);
    case 4: return n.at<void>(n.p.pool[2]);
    case 6: return n.at<void>(n.p.pool[3]);
    case 8: return n.at<void>(n.p.up[2]);
    case 10: return n.at<void>(n.p.up[1]);
    case 12: return n.at<void>(n.p.up[0]);
    default: return n.at<void>(n.p.act[l - 1]);
  }
}

pf_status conv_layer(const Net& n, const float* params, int l) {
  const LayerDef& L = kLayers[l];
  const int lv = L.level;
  const bool last = (l == kNL - 1);
  SG_CUDA(conv(n, L.cin, L.cout, layer_input(n, l), n.at<void>(n.p.wf[l]), params + b_off(l),
               L.relu, last ? nullptr : n.at<void>(n.p.act[l]),
               last ? n.at<float>(n.p.y32) : nullptr, n.dim(lv, 0), n.dim(lv, 1), n.dim(lv, 2)));
  return PF_OK;
}

// Input mode = number of previous states: 8 channels = U^n alone (output unit
// out_scale); 16 = [U^n; U^{n-1}] and 24 = [U^n; U^{n-1}; U^{n-2}] (the network
// sees U^n and the increments in units of the RMS of the last one; the output
// unit is out_scale times that RMS on top of linear extrapolation, and
// out_scale times the RMS of the second difference, floored at 1e-3 of the
// increment unit, on top of quadratic extrapolation).
int in_mode(int n_in) { return n_in / kNF - 1; }
bool n_in_ok(int n_in) { return n_in == kNF || n_in == 2 * kNF || n_in == 3 * kNF; }

pf_status forward(const Net& n, const float* params, const float* x, int n_in, float out_scale) {
  const Plan& p = n.p;
  const int64_t V0 = p.V[0] / p.B;
  const int mode = in_mode(n_in);
  SG_CUDA(pf::launch_incr_scale(x, kNF, p.B, V0, out_scale, mode, n.at<double>(p.sigp),
                                kSigBlocks, n.at<float>(p.sig), n.at<float>(p.sigo), n.s));
  SG_CUDA(pf::launch_planar_to_ndhwc(x, n_in, kCin0, p.B, V0, mode, n.at<float>(p.sig),
                                     n.at<void>(p.x16), n.s));
  pf_status st;
  for (int l = 0; l < kNL; ++l) {
    if (l == 2 || l == 4 || l == 6) {  // pool the previous level's last activation
      const int lv = kLayers[l].level;
      SG_CUDA(pf::launch_pool(n.at<void>(p.act[l - 1]), p.B, n.dim(lv - 1, 0), n.dim(lv - 1, 1),
                              n.dim(lv - 1, 2), kC, n.at<void>(p.pool[lv]), n.s));
    }
    if (l == 8 || l == 10 || l == 12) {  // upsample the coarser output and add the skip
      const int lv = kLayers[l].level;
      const int skip = (lv == 2) ? 5 : (lv == 1) ? 3 : 1;
      SG_CUDA(pf::launch_up_add(n.at<void>(p.act[l - 1]), n.at<void>(p.act[skip]), p.B,
                                n.dim(lv, 0), n.dim(lv, 1), n.dim(lv, 2), kC, n.at<void>(p.up[lv]),
                                n.s));
    }
    if ((st = conv_layer(n, params, l)) != PF_OK) return st;
  }
  return PF_OK;
}

// gradient of layer l's output is in dy (masked here if the layer has a ReLU);
// writes dW, db into grad and, if dx != nullptr, the input gradient.
pf_status backward_layer(const Net& n, int l, void* dy, void* dx, float* grad) {
  const LayerDef& L = kLayers[l];
  const int lv = L.level;
  const int d = n.dim(lv, 0), h = n.dim(lv, 1), w = n.dim(lv, 2);
  const int64_t nvox = (int64_t)n.p.B * d * h * w;
  if (L.relu) SG_CUDA(pf::launch_relu_mask(dy, n.at<void>(n.p.act[l]), nvox * L.cout, n.s));
  if (n.tc && pf::wgrad_tc_shape_ok(n.p.B, d, h, w)) {
    SG_CUDA(pf::launch_wgrad_tc(L.cin, L.cout, layer_input(n, l), dy, n.at<float>(n.p.part),
                                grad + w_off(l), n.p.B, d, h, w, n.at<int>(n.p.err), n.s));
  } else {
    const int blocks = pf::conv_wgrad_blocks(n.p.B, d, h, w, wgrad_blocks());
    SG_CUDA(pf::launch_conv3d_wgrad(L.cin, L.cout, layer_input(n, l), dy, n.at<float>(n.p.part),
                                    grad + w_off(l), n.p.B, d, h, w, blocks, n.s));
  }
  // (the weight-gradient partials are summed by now: their buffer is free)
  SG_CUDA(pf::launch_bias_grad(dy, L.cout, nvox, grad + b_off(l), n.at<float>(n.p.part), n.s));
  if (dx) SG_CUDA(conv(n, L.cout, L.cin, dy, n.at<void>(n.p.wb[l]), nullptr, 0, dx, nullptr, d, h, w));
  return PF_OK;
}

pf_status backward(const Net& n, float* grad) {
  const Plan& p = n.p;
  auto G = [&](int lv, int k) { return n.at<void>(p.g[lv][k]); };
  auto down = [&](int lv_fine, void* g_fine, void* g_coarse) {
    return pf::launch_down_sum(g_fine, p.B, n.dim(lv_fine, 0), n.dim(lv_fine, 1),
                               n.dim(lv_fine, 2), kC, g_coarse, n.s);
  };
  auto pool_back = [&](int lv_fine, void* g_coarse, void* acc) {
    return pf::launch_pool_back_add(g_coarse, p.B, n.dim(lv_fine, 0), n.dim(lv_fine, 1),
                                    n.dim(lv_fine, 2), kC, acc, n.s);
  };
  pf_status st;
#define STEP(x)                              \
  do {                                       \
    if ((st = (x)) != PF_OK) return st;      \
  } while (0)
#define CU(x) SG_CUDA(x)
  STEP(backward_layer(n, 14, n.at<void>(p.gy), G(0, 0), grad));
  STEP(backward_layer(n, 13, G(0, 0), G(0, 1), grad));
  STEP(backward_layer(n, 12, G(0, 1), G(0, 2), grad));  // G(0,2): d up0 = d skip0
  CU(down(0, G(0, 2), G(1, 0)));                         // d act11
  STEP(backward_layer(n, 11, G(1, 0), G(1, 1), grad));
  STEP(backward_layer(n, 10, G(1, 1), G(1, 2), grad));  // G(1,2): d up1 = d skip1
  CU(down(1, G(1, 2), G(2, 0)));                         // d act9
  STEP(backward_layer(n, 9, G(2, 0), G(2, 1), grad));
  STEP(backward_layer(n, 8, G(2, 1), G(2, 2), grad));   // G(2,2): d up2 = d skip2
  CU(down(2, G(2, 2), G(3, 0)));                         // d act7
  STEP(backward_layer(n, 7, G(3, 0), G(3, 1), grad));
  STEP(backward_layer(n, 6, G(3, 1), G(3, 2), grad));   // d pool3
  CU(pool_back(2, G(3, 2), G(2, 2)));                    // d act5 = skip + pool back
  STEP(backward_layer(n, 5, G(2, 2), G(2, 0), grad));
  STEP(backward_layer(n, 4, G(2, 0), G(2, 1), grad));   // d pool2
  CU(pool_back(1, G(2, 1), G(1, 2)));                    // d act3
  STEP(backward_layer(n, 3, G(1, 2), G(1, 0), grad));
  STEP(backward_layer(n, 2, G(1, 0), G(1, 1), grad));   // d pool1
  CU(pool_back(0, G(1, 1), G(0, 2)));                    // d act1
  STEP(backward_layer(n, 1, G(0, 2), G(0, 0), grad));
  STEP(backward_layer(n, 0, G(0, 0), nullptr, grad));
#undef STEP
#undef CU
  return PF_OK;
}

}  // namespace

extern "C" {

pf_status pf_surrogate_param_count(int64_t* n) {
  if (!n) return PF_ERR_ARG;
  *n = param_count();
  return PF_OK;
}

pf_status pf_surrogate_workspace(int batch, int d, int h, int w, int training, size_t* bytes) {
  if (!bytes || !dims_ok(batch, d, h, w)) return PF_ERR_ARG;
  *bytes = make_plan(batch, d, h, w, training != 0).total;
  return PF_OK;
}

pf_status pf_surrogate_predict(const float* params, float out_scale, const float* x, int n_in,
                               float* out, int batch, int d, int h, int w, void* ws, size_t bytes,
                               void* stream) {
  if (!params || !x || !out || !ws || !dims_ok(batch, d, h, w) || !scale_ok(out_scale) ||
      !n_in_ok(n_in))
    return PF_ERR_ARG;
  const Plan p = make_plan(batch, d, h, w, false);
  if (bytes < p.total || (uintptr_t)ws % 256) return PF_ERR_ARG;
  Net n{p, (char*)ws, (cudaStream_t)stream, true};
  pf_status st = clear_err(n);
  if (st != PF_OK || (st = convert_all(n, params, false)) != PF_OK) return st;
  if ((st = forward(n, params, x, n_in, out_scale)) != PF_OK) return st;
  SG_CUDA(pf::launch_ndhwc_to_planar_add(n.at<float>(p.y32), kCout, kNF, batch,
                                         (int64_t)d * h * w, x, n_in, in_mode(n_in),
                                         n.at<float>(p.sigo), out, n.s));
  return check_err(n);
}

pf_status pf_surrogate_train_step(float* params, float out_scale, float* adam_m, float* adam_v,
                                  int step, double lr, const float* x, int n_in, const float* y,
                                  double stiff, int batch, int d, int h, int w, void* ws,
                                  size_t bytes, void* stream, double* loss) {
  if (!params || !adam_m || !adam_v || !x || !y || !ws || step < 1 || !(lr > 0) ||
      !(stiff >= 0) || !isfinite(stiff) ||
      !dims_ok(batch, d, h, w) || !scale_ok(out_scale) || !n_in_ok(n_in))
    return PF_ERR_ARG;
  const Plan p = make_plan(batch, d, h, w, true);
  if (bytes < p.total || (uintptr_t)ws % 256) return PF_ERR_ARG;
  Net n{p, (char*)ws, (cudaStream_t)stream, true};
  pf_status st = clear_err(n);
  if (st != PF_OK || (st = convert_all(n, params, true)) != PF_OK) return st;
  if ((st = forward(n, params, x, n_in, out_scale)) != PF_OK) return st;
  const int64_t V = (int64_t)d * h * w;
  const float scale = (float)(1.0 / ((double)batch * V * kNF));
  SG_CUDA(pf::launch_mse(n.at<float>(p.y32), kCout, kNF, n_in, batch, d, h, w, x, y,
                         in_mode(n_in), n.at<float>(p.sigo), (float)stiff, scale,
                         n.at<float>(p.res), n.at<float>(p.resq), n.at<void>(p.gy),
                         n.at<double>(p.msep), n.at<double>(p.loss), n.s));
  float* grad = n.at<float>(p.grad);
  if ((st = backward(n, grad)) != PF_OK) return st;
  SG_CUDA(pf::launch_adam(params, adam_m, adam_v, grad, param_count(), (float)lr, 0.9f, 0.999f,
                          1e-8f, step, n.s));
  if (loss) {
    SG_CUDA(cudaMemcpyAsync(loss, n.at<double>(p.loss), sizeof(double), cudaMemcpyDeviceToHost,
                            n.s));
    return check_err(n);
  }
  return PF_OK;
}

pf_status pf_surrogate_loss_grad(const float* params, float out_scale, const float* x, int n_in,
                                 const float* y, double stiff, int batch, int d, int h, int w,
                                 void* ws, size_t bytes, void* stream, double* loss,
                                 float* grad) {
  if (!params || !x || !y || !ws || !grad || !dims_ok(batch, d, h, w) || !scale_ok(out_scale) ||
      !(stiff >= 0) || !isfinite(stiff) ||
      !n_in_ok(n_in))
    return PF_ERR_ARG;
  const Plan p = make_plan(batch, d, h, w, true);
  if (bytes < p.total || (uintptr_t)ws % 256) return PF_ERR_ARG;
  Net n{p, (char*)ws, (cudaStream_t)stream, true};
  pf_status st = clear_err(n);
  if (st != PF_OK || (st = convert_all(n, params, true)) != PF_OK) return st;
  if ((st = forward(n, params, x, n_in, out_scale)) != PF_OK) return st;
  const int64_t V = (int64_t)d * h * w;
  const float scale = (float)(1.0 / ((double)batch * V * kNF));
  SG_CUDA(pf::launch_mse(n.at<float>(p.y32), kCout, kNF, n_in, batch, d, h, w, x, y,
                         in_mode(n_in), n.at<float>(p.sigo), (float)stiff, scale,
                         n.at<float>(p.res), n.at<float>(p.resq), n.at<void>(p.gy),
                         n.at<double>(p.msep), n.at<double>(p.loss), n.s));
  if ((st = backward(n, grad)) != PF_OK) return st;
  if (loss) {
    SG_CUDA(cudaMemcpyAsync(loss, n.at<double>(p.loss), sizeof(double), cudaMemcpyDeviceToHost,
                            n.s));
    return check_err(n);
  }
  return PF_OK;
}

pf_status pf_conv3d_check(int mode, int cin, int cout, int d, int h, int w, const float* x,
                          const float* wt, const float* bias, const float* dy, float* out,
                          void* ws, size_t bytes, void* stream) {
  // Single-layer probe of the convolution kernels for parity tests: planar FP32
  // in and out ([c][d][h][w], one sample), weights [27][c_out][c_in] FP32.
  // mode 0: out = conv(x) + bias; 1: out = conv^T(dy); 2: out = [dW (27 c_out c_in), db];
  // modes 0, 1 and 2 take the tcgen05 kernels where the shape allows, 3, 4 and 6
  // are 0, 1 and 2 on the mma.sync kernels; 5 is mode 0 on the tcgen05 kernel with
  // no input copies issued (the bounded pipeline waits must expire: PF_ERR_TIMEOUT).
  const bool ok_c = (cin == 16 && cout == 32) || (cin == 32 && cout == 32) ||
                    (cin == 32 && cout == 16);
  if (!ok_c || mode < 0 || mode > 6 || !x || !wt || !out || !ws || d % 2 || h % 8 || w % 8 ||
      d < 2 || h < 8 || w < 8)
    return PF_ERR_ARG;
  const int64_t V = (int64_t)d * h * w;
  size_t need = al(2 * V * cin) + al(2 * V * cout) + 2 * al(2 * 27 * cin * cout) + al(4 * V * kC) +
                al(4 * part_floats(cin, cout)) + al(sizeof(int));
  if (bytes < need || (mode == 1 || mode == 2 || mode == 4 || mode == 6) && !dy ||
      (uintptr_t)ws % 256)
    return PF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  char* p = (char*)ws;
  void* xb = p;
  p += al(2 * V * cin);
  void* db16 = p;
  p += al(2 * V * cout);
  void* wf = p;
  p += al(2 * 27 * cin * cout);
  void* wb = p;
  p += al(2 * 27 * cin * cout);
  float* y32 = (float*)p;
  p += al(4 * V * kC);
  float* part = (float*)p;
  p += al(4 * part_floats(cin, cout));
  int* err = (int*)p;
  const bool tc = (mode == 0 || mode == 1 || mode == 5) && pf::conv3d_tc_shape_ok(1, d, h, w);
  const int selftest = mode == 5;
  if (mode == 5 && !tc) return PF_ERR_ARG;
  auto run = [&](int ci, int co, const void* in, const void* wts, const float* bs) {
    return tc ? pf::launch_conv3d_tc(ci, co, in, wts, bs, 0, nullptr, y32, 1, d, h, w, err, s,
                                     selftest)
              : pf::launch_conv3d(ci, co, in, wts, bs, 0, nullptr, y32, 1, d, h, w, conv_grid(), s);
  };
  SG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  SG_CUDA(pf::launch_convert_weights(wt, cin, cout, wf, wb, s));
  SG_CUDA(pf::launch_planar_to_ndhwc(x, cin, cin, 1, V, 0, nullptr, xb, s));
  if (mode == 0 || mode == 3 || mode == 5) {
    SG_CUDA(run(cin, cout, xb, wf, bias));
    SG_CUDA(pf::launch_ndhwc_to_planar_add(y32, cout, cout, 1, V, nullptr, 0, 0, nullptr, out, s));
  } else {
    SG_CUDA(pf::launch_planar_to_ndhwc(dy, cout, cout, 1, V, 0, nullptr, db16, s));
    if (mode == 1 || mode == 4) {
      SG_CUDA(run(cout, cin, db16, wb, nullptr));
      SG_CUDA(pf::launch_ndhwc_to_planar_add(y32, cin, cin, 1, V, nullptr, 0, 0, nullptr, out, s));
    } else {
      if (mode == 2 && pf::wgrad_tc_shape_ok(1, d, h, w)) {
        SG_CUDA(pf::launch_wgrad_tc(cin, cout, xb, db16, part, out, 1, d, h, w, err, s));
      } else {
        const int blocks = pf::conv_wgrad_blocks(1, d, h, w, wgrad_blocks());
        SG_CUDA(pf::launch_conv3d_wgrad(cin, cout, xb, db16, part, out, 1, d, h, w, blocks, s));
      }
      SG_CUDA(pf::launch_bias_grad(db16, cout, V, out + 27 * cin * cout, part, s));
    }
  }
  int e = 0;
  SG_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SG_CUDA(cudaStreamSynchronize(s));
  return e ? PF_ERR_TIMEOUT : PF_OK;
}

}  // extern "C"
