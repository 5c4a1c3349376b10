// C ABI of the differentiable unrolled mean-shift steps (see k_unroll.cu for
// the kernels and the adjoint formulas), in FP32 and, for checking gradients,
// FP64 (the *_f64 entry points).
#include <math.h>
#include <string.h>

#include "../../include/fms.h"
#include "fms_internal.cuh"


using namespace fms;

namespace {

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

bool valid(int32_t B, int64_t n, int64_t m, int32_t d, int32_t T, int32_t k) {
  return B >= 1 && n >= 1 && m >= 1 && n <= INT32_MAX && m <= INT32_MAX && d >= 1 && d <= 32 &&
         T >= 1 && k >= 1 && (int64_t)B * n <= INT32_MAX && (int64_t)B * m <= INT32_MAX;
}

int sm_count() {
  int dev = 0, s = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return s;
}

// Chunks so that (sets x groups of 32 outputs x chunks) ~ 8 tasks per resident warp.
void chunks(int64_t groups, int64_t len, int sms, int* C, int* L) {
  const int64_t target = (int64_t)(sms > 0 ? sms : 1) * 16 * 8;
  int64_t c = (target + groups - 1) / groups;
  if (c < 1) c = 1;
  if (c > (len + 63) / 64) c = (len + 63) / 64;
  if (c < 1) c = 1;
  int64_t l = (len + c - 1) / c;
  *C = (int)((len + l - 1) / l);
  *L = (int)l;
}

// rows padded to 4, 8, 16 or 32 floats (the kernels know the width at compile time)
int padded_width(int d) { return d <= 4 ? 4 : (d <= 8 ? 8 : (d <= 16 ? 16 : 32)); }

UGeom geom(int32_t B, int64_t n, int64_t m, int32_t d) {
  UGeom g{};
  g.B = B;
  g.n = (int)n;
  g.m = (int)m;
  g.d = d;
  g.DP = padded_width(d);
  const int sms = sm_count();
  // seed-major passes: groups of 32 seeds; point-major pass: 64 points (32 at DP = 32)
  const int ppw = g.DP <= 16 ? 64 : 32;
  chunks((int64_t)B * ((m + 31) / 32), n, sms, &g.Cp, &g.Lp);
  chunks((int64_t)B * ((n + ppw - 1) / ppw), m, sms, &g.Cs, &g.Ls);
  return g;
}

int grid_blocks() {
  const int s = sm_count();
  return (s > 0 ? s : 1) * 8;
}

int n_ckpt(int32_t T, int32_t k) { return (T + k - 1) / k; }

struct FwdLayout {
  size_t Xp, Ya, Yb, part, rlist, status, total;
};
FwdLayout fwd_layout(const UGeom& g, size_t es) {
  FwdLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o += a256(b > 0 ? b : 1);
    return at;
  };
  L.Xp = take((size_t)g.B * g.n * g.DP * es);
  L.Ya = take((size_t)g.B * g.m * g.DP * es);
  L.Yb = take((size_t)g.B * g.m * g.DP * es);
  L.part = take((size_t)g.B * g.Cp * g.m * (g.DP + 1) * es);
  L.rlist = take(((size_t)g.B * g.m + 1) * 4);   // rescue list, then its count
  L.status = take(64);   // kStTimeout if a staged-row wait gave up
  L.total = o;
  return L;
}

struct BwdLayout {
  size_t Xp, seg, Ga, Gb, part_s, part_p, SD, dh_part, dXp, dh, rlist, status, total;
};
BwdLayout bwd_layout(const UGeom& g, int32_t k, size_t es) {
  BwdLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o += a256(b > 0 ? b : 1);
    return at;
  };
  const size_t rowsY = (size_t)g.B * g.m;
  L.Xp = take((size_t)g.B * g.n * g.DP * es);
  L.seg = take((size_t)k * rowsY * g.DP * es);   // recomputed positions inside a segment
  L.Ga = take(rowsY * g.DP * es);
  L.Gb = take(rowsY * g.DP * es);
  L.part_s = take((size_t)g.B * g.Cp * g.m * (g.DP + 1) * es);
  L.part_p = take((size_t)g.B * g.Cs * g.n * g.DP * es);
  L.SD = take(rowsY * (2 * g.DP + 4) * es);
  L.dh_part = take(rowsY * es);
  L.dXp = take((size_t)g.B * g.n * g.DP * es);
  L.dh = take((size_t)g.B * 8);
  L.rlist = take((rowsY + 1) * 4);
  L.status = take(64);
  L.total = o;
  return L;
}

// The checkpoint buffer: positions Y_t for t = 0, k, 2k, .. and Y_T (rows of
// DP values), then W_t and the weight shift of every update t < T (one value
// per seed each), so the backward recomputes only the positions between
// checkpoints.
struct CkptLayout {
  size_t pos, W, Sh, total;
};
CkptLayout ckpt_layout(int32_t B, int64_t m, int32_t d, int32_t T, int32_t k, size_t es) {
  CkptLayout C{};
  const size_t rowsY = (size_t)B * m;
  C.pos = 0;
  C.W = (size_t)(n_ckpt(T, k) + 1) * rowsY * padded_width(d) * es;
  C.Sh = C.W + (size_t)T * rowsY * es;
  C.total = C.Sh + (size_t)T * rowsY * es;
  return C;
}

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

}  // namespace

namespace {

template <typename E>
fms_status forward_impl(const E* points, const E* seeds0, int32_t B, int64_t n,
                                int64_t m, int32_t d, E h, int32_t T, int32_t k,
                                E* out_seeds, void* ckpt, size_t ckpt_bytes, void* ws,
                                size_t ws_bytes, void* stream) {
  if (!points || !seeds0 || !out_seeds || !valid(B, n, m, d, T, k) || !(h > 0) || !isfinite(h))
    return FMS_ERR_INVALID_ARG;
  if (!ws || !ckpt) return FMS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const UGeom g = geom(B, n, m, d);
  const FwdLayout L = fwd_layout(g, sizeof(E));
  if (ws_bytes < L.total || ckpt_bytes < ckpt_layout(B, m, d, T, k, sizeof(E)).total ||
      (reinterpret_cast<uintptr_t>(ws) & 255u) || (reinterpret_cast<uintptr_t>(ckpt) & 15u))
    return FMS_ERR_WORKSPACE;
  E* Xp = at<E>(ws, L.Xp);
  E* Ya = at<E>(ws, L.Ya);
  E* Yb = at<E>(ws, L.Yb);
  E* part = at<E>(ws, L.part);
  int32_t* rlist = at<int32_t>(ws, L.rlist);
  int32_t* rcount = rlist + (size_t)B * m;
  uint32_t* status = at<uint32_t>(ws, L.status);
  const CkptLayout CL = ckpt_layout(B, m, d, T, k, sizeof(E));
  E* C = at<E>(ckpt, CL.pos);
  E* Wh = at<E>(ckpt, CL.W);
  E* Shh = at<E>(ckpt, CL.Sh);
  const size_t rowsY = (size_t)B * m;
  const E c = (E)(1.4426950408889634 / (2.0 * (double)h * (double)h));
  const int grid = grid_blocks();
  if (unroll_pack_rows<E>(points, (int64_t)B * n, d, g.DP, Xp, st) != cudaSuccess ||
      unroll_pack_rows<E>(seeds0, (int64_t)rowsY, d, g.DP, Ya, st) != cudaSuccess ||
      cudaMemsetAsync(rcount, 0, 4, st) != cudaSuccess ||
      cudaMemsetAsync(status, 0, 64, st) != cudaSuccess)
    return FMS_ERR_CUDA;
  for (int t = 0; t < T; ++t) {
    if (t % k == 0 &&
        cudaMemcpyAsync(C + (size_t)(t / k) * rowsY * g.DP, Ya, rowsY * g.DP * sizeof(E),
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return FMS_ERR_CUDA;
    if (unroll_fwd_step<E>(Xp, Ya, g, c, part, Yb, Wh + (size_t)t * rowsY, Shh + (size_t)t * rowsY,
                           rlist, rcount, grid, status, st) != cudaSuccess)
      return FMS_ERR_CUDA;
    E* tmp = Ya;
    Ya = Yb;
    Yb = tmp;
  }
  if (cudaMemcpyAsync(C + (size_t)n_ckpt(T, k) * rowsY * g.DP, Ya, rowsY * g.DP * sizeof(E),
                      cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      unroll_unpack_rows<E>(Ya, (int64_t)rowsY, d, g.DP, out_seeds, st) != cudaSuccess)
    return FMS_ERR_CUDA;
  return FMS_OK;
}

template <typename E>
fms_status backward_impl(const E* points, int32_t B, int64_t n, int64_t m, int32_t d,
                                 E h, int32_t T, int32_t k, const void* ckpt,
                                 size_t ckpt_bytes, const E* grad_out, E* grad_points,
                                 E* grad_seeds0, double* grad_h, void* ws, size_t ws_bytes,
                                 void* stream) {
  if (!points || !grad_out || !grad_points || !grad_seeds0 || !grad_h ||
      !valid(B, n, m, d, T, k) || !(h > 0) || !isfinite(h))
    return FMS_ERR_INVALID_ARG;
  if (!ws || !ckpt) return FMS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const UGeom g = geom(B, n, m, d);
  const BwdLayout L = bwd_layout(g, k, sizeof(E));
  if (ws_bytes < L.total || ckpt_bytes < ckpt_layout(B, m, d, T, k, sizeof(E)).total ||
      (reinterpret_cast<uintptr_t>(ws) & 255u) || (reinterpret_cast<uintptr_t>(ckpt) & 15u))
    return FMS_ERR_WORKSPACE;
  E* Xp = at<E>(ws, L.Xp);
  E* seg = at<E>(ws, L.seg);
  int32_t* rlist = at<int32_t>(ws, L.rlist);
  int32_t* rcount = rlist + (size_t)B * m;
  E* Ga = at<E>(ws, L.Ga);
  E* Gb = at<E>(ws, L.Gb);
  E* part_s = at<E>(ws, L.part_s);
  E* part_p = at<E>(ws, L.part_p);
  E* SD = at<E>(ws, L.SD);
  uint32_t* status = at<uint32_t>(ws, L.status);
  E* dh_part = at<E>(ws, L.dh_part);
  E* dXp = at<E>(ws, L.dXp);
  double* dh = at<double>(ws, L.dh);
  const CkptLayout CL = ckpt_layout(B, m, d, T, k, sizeof(E));
  const E* Ck = static_cast<const E*>(ckpt);
  const E* Wh = Ck + CL.W / sizeof(E);
  const E* Shh = Ck + CL.Sh / sizeof(E);
  const size_t rowsY = (size_t)B * m;
  const size_t rowY = rowsY * g.DP;
  const double hd = (double)h;
  const E c = (E)(1.4426950408889634 / (2.0 * hd * hd));
  const E inv_h2 = (E)(1.0 / (hd * hd)), inv_h3 = (E)(1.0 / (hd * hd * hd));
  const int grid = grid_blocks();
  if (unroll_pack_rows<E>(points, (int64_t)B * n, d, g.DP, Xp, st) != cudaSuccess ||
      unroll_pack_rows<E>(grad_out, (int64_t)rowsY, d, g.DP, Ga, st) != cudaSuccess ||
      cudaMemsetAsync(dXp, 0, (size_t)B * n * g.DP * sizeof(E), st) != cudaSuccess ||
      cudaMemsetAsync(dh, 0, (size_t)B * 8, st) != cudaSuccess ||
      cudaMemsetAsync(rcount, 0, 4, st) != cudaSuccess ||
      cudaMemsetAsync(status, 0, 64, st) != cudaSuccess)
    return FMS_ERR_CUDA;
  E* G = Ga;
  E* Gp = Gb;
  for (int s = n_ckpt(T, k) - 1; s >= 0; --s) {
    const int t0 = s * k;
    const int len = (t0 + k <= T) ? k : T - t0;
    // positions of the segment: Y_t0 and Y_{t0+len} are checkpoints (the last
    // is Y_T for the final segment); Y_{t0+1} .. Y_{t0+len-1} are recomputed
    // into seg (W and the shifts of every update were stored by the forward)
    auto pos = [&](int u) -> const E* {
      if (u == 0) return Ck + (size_t)s * rowY;
      if (u == len) return Ck + (size_t)(s + 1) * rowY;
      return seg + (size_t)(u - 1) * rowY;
    };
    for (int u = 0; u + 1 < len; ++u)
      if (unroll_fwd_step<E>(Xp, pos(u), g, c, part_s, seg + (size_t)u * rowY, nullptr, nullptr,
                             rlist, rcount, grid, status, st) != cudaSuccess)
        return FMS_ERR_CUDA;
    for (int u = len - 1; u >= 0; --u) {
      const size_t t = (size_t)(t0 + u);
      if (unroll_bwd_step<E>(Xp, pos(u), pos(u + 1), G, Wh + t * rowsY, Shh + t * rowsY, g, c,
                             inv_h2, inv_h3, part_s, part_p, SD, dh_part, Gp, dXp, dh, grid,
                             status, st) != cudaSuccess)
        return FMS_ERR_CUDA;
      E* tmp = G;
      G = Gp;
      Gp = tmp;
    }
  }
  if (unroll_unpack_rows<E>(G, (int64_t)rowsY, d, g.DP, grad_seeds0, st) != cudaSuccess ||
      unroll_unpack_rows<E>(dXp, (int64_t)B * n, d, g.DP, grad_points, st) != cudaSuccess ||
      cudaMemcpyAsync(grad_h, dh, (size_t)B * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return FMS_ERR_CUDA;
  return FMS_OK;
}

}  // namespace

extern "C" {

size_t fms_unrolled_ckpt_size(int32_t B, int64_t n, int64_t m, int32_t d, int32_t T, int32_t k) {
  if (!valid(B, n, m, d, T, k)) return 0;
  return ckpt_layout(B, m, d, T, k, 4).total;
}

size_t fms_unrolled_workspace_size(int32_t B, int64_t n, int64_t m, int32_t d, int32_t T,
                                   int32_t k) {
  if (!valid(B, n, m, d, T, k)) return 0;
  const UGeom g = geom(B, n, m, d);
  const size_t f = fwd_layout(g, 4).total, b = bwd_layout(g, k, 4).total;
  return f > b ? f : b;
}

fms_status fms_unrolled_forward(const float* points, const float* seeds0, int32_t B, int64_t n,
                                int64_t m, int32_t d, float h, int32_t T, int32_t k,
                                float* out_seeds, void* ckpt, size_t ckpt_bytes, void* ws,
                                size_t ws_bytes, void* stream) {
  return forward_impl<float>(points, seeds0, B, n, m, d, h, T, k, out_seeds, ckpt, ckpt_bytes, ws,
                             ws_bytes, stream);
}

fms_status fms_unrolled_backward(const float* points, int32_t B, int64_t n, int64_t m, int32_t d,
                                 float h, int32_t T, int32_t k, const void* ckpt,
                                 size_t ckpt_bytes, const float* grad_out, float* grad_points,
                                 float* grad_seeds0, double* grad_h, void* ws, size_t ws_bytes,
                                 void* stream) {
  return backward_impl<float>(points, B, n, m, d, h, T, k, ckpt, ckpt_bytes, grad_out,
                              grad_points, grad_seeds0, grad_h, ws, ws_bytes, stream);
}

size_t fms_unrolled_ckpt_size_f64(int32_t B, int64_t n, int64_t m, int32_t d, int32_t T,
                                  int32_t k) {
  if (!valid(B, n, m, d, T, k)) return 0;
  return ckpt_layout(B, m, d, T, k, 8).total;
}

size_t fms_unrolled_workspace_size_f64(int32_t B, int64_t n, int64_t m, int32_t d, int32_t T,
                                       int32_t k) {
  if (!valid(B, n, m, d, T, k)) return 0;
  const UGeom g = geom(B, n, m, d);
  const size_t f = fwd_layout(g, 8).total, b = bwd_layout(g, k, 8).total;
  return f > b ? f : b;
}

fms_status fms_unrolled_forward_f64(const double* points, const double* seeds0, int32_t B,
                                    int64_t n, int64_t m, int32_t d, double h, int32_t T,
                                    int32_t k, double* out_seeds, void* ckpt, size_t ckpt_bytes,
                                    void* ws, size_t ws_bytes, void* stream) {
  return forward_impl<double>(points, seeds0, B, n, m, d, h, T, k, out_seeds, ckpt, ckpt_bytes,
                              ws, ws_bytes, stream);
}

fms_status fms_unrolled_backward_f64(const double* points, int32_t B, int64_t n, int64_t m,
                                     int32_t d, double h, int32_t T, int32_t k, const void* ckpt,
                                     size_t ckpt_bytes, const double* grad_out,
                                     double* grad_points, double* grad_seeds0, double* grad_h,
                                     void* ws, size_t ws_bytes, void* stream) {
  return backward_impl<double>(points, B, n, m, d, h, T, k, ckpt, ckpt_bytes, grad_out,
                               grad_points, grad_seeds0, grad_h, ws, ws_bytes, stream);
}

}  // extern "C"
