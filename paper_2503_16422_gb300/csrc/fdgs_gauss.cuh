// Per-Gaussian stage of the 4D Gaussian rasterizer: 4D covariance from the scale and the
// left/right quaternion pair (Sec. 3), slice at time t (Eq. 1) with the temporal weight
// (Eq. 3), EWA projection to a 2D conic, tile radius, SH colour; and its reverse.
//
// Numerical form (mathematically identical to Eq. 1, better conditioned in float32):
// with M = R diag(s) (so Sigma = M M^T), m_t = row t of M, m^ = m_t/|m_t| and M_x the xyz
// rows, Sigma_t = |m_t|^2, Sigma_xt = M_x m_t and
//   Sigma_xyz|t = M_x (I - m^ m^T) M_x^T = N N^T,  N = M_x - w m^T,  w = M_x m^,
//   mu_xyz|t    = mu_xyz + w (t - mu_t) / |m_t|.
// The 2D covariance is then (T N)(T N)^T + 0.3 I with T = J R_view, so it is PSD by
// construction; its determinant uses the Lagrange identity (sum of squared 2x2 minors).
#pragma once
#include "fdgs_common.cuh"

namespace fdgs {

struct GaussState {
  float qn_l[4], qn_r[4], inv_l, inv_r;   // normalised quaternions, 1/|q|
  float Lm[16], Rm[16], R[16];            // left/right isoclinic factors, R = Lm Rm
  float s[4], M[16];                      // scales, M = R diag(s)
  float nt2, nt, mh[4], w[3], N[12];      // Sigma_t, |m_t|, m^, w, N (3x4)
  float dt, p, sig, a;                    // t - mu_t, temporal weight, sigmoid(o), opacity
  float mu3[3], xc[3], iz, xr, yr, xz, yz;
  bool clx, cly;                          // Jacobian clamp active on x / y
  float T2[6], P[8];                      // T = J R_view (2x3), P = T N (2x4)
  float c00, c01, c11, det;               // 2D covariance (dilated) and determinant
  float dn[3], dlen;                      // view direction
  float raw[3];                           // colour before the clamp at 0
};

__device__ __forceinline__ void quat_unit(float4 q, float o[4], float &inv) {
  float n2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  inv = rsqrtf(n2);
  o[0] = q.x * inv; o[1] = q.y * inv; o[2] = q.z * inv; o[3] = q.w * inv;
}

// v -> q v (Hamilton product), q = (a, b, c, d)
__device__ __forceinline__ void left_mat(const float q[4], float L[16]) {
  const float a = q[0], b = q[1], c = q[2], d = q[3];
  L[0] = a;  L[1] = -b; L[2] = -c;  L[3] = -d;
  L[4] = b;  L[5] = a;  L[6] = -d;  L[7] = c;
  L[8] = c;  L[9] = d;  L[10] = a;  L[11] = -b;
  L[12] = d; L[13] = -c; L[14] = b; L[15] = a;
}
// v -> v q (Hamilton product), q = (p, q, r, s)
__device__ __forceinline__ void right_mat(const float q[4], float Rr[16]) {
  const float p = q[0], x = q[1], r = q[2], s = q[3];
  Rr[0] = p;  Rr[1] = -x; Rr[2] = -r;  Rr[3] = -s;
  Rr[4] = x;  Rr[5] = p;  Rr[6] = s;   Rr[7] = -r;
  Rr[8] = r;  Rr[9] = -s; Rr[10] = p;  Rr[11] = x;
  Rr[12] = s; Rr[13] = r; Rr[14] = -x; Rr[15] = p;
}

// Real spherical harmonics without the Condon-Shortley phase, k = l^2 + l + m, degree <= 3.
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.4886025119029199f;                 // sqrt(3/(4 pi))
constexpr float kSH2a = 1.0925484305920792f;                // 1/2 sqrt(15/pi)
constexpr float kSH2b = 0.31539156525252005f;               // 1/4 sqrt(5/pi)
constexpr float kSH2c = 0.5462742152960396f;                // 1/4 sqrt(15/pi)
constexpr float kSH3a = 0.5900435899266435f;                // 1/4 sqrt(35/(2 pi))
constexpr float kSH3b = 2.890611442640554f;                 // 1/2 sqrt(105/pi)
constexpr float kSH3c = 0.4570457994644658f;                // 1/4 sqrt(21/(2 pi))
constexpr float kSH3d = 0.3731763325901154f;                // 1/4 sqrt(7/pi)
constexpr float kSH3e = 1.445305721320277f;                 // 1/4 sqrt(105/pi)

__device__ __forceinline__ void sh_eval(int deg, float x, float y, float z, float Y[16]) {
  Y[0] = kSH0;
  if (deg < 1) return;
  Y[1] = kSH1 * y; Y[2] = kSH1 * z; Y[3] = kSH1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kSH2a * x * y; Y[5] = kSH2a * y * z; Y[6] = kSH2b * (3.f * zz - 1.f);
  Y[7] = kSH2a * x * z; Y[8] = kSH2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = kSH3a * y * (3.f * xx - yy); Y[10] = kSH3b * x * y * z;
  Y[11] = kSH3c * y * (5.f * zz - 1.f); Y[12] = kSH3d * z * (5.f * zz - 3.f);
  Y[13] = kSH3c * x * (5.f * zz - 1.f); Y[14] = kSH3e * z * (xx - yy);
  Y[15] = kSH3a * x * (xx - 3.f * yy);
}

// Gradient of sum_k g[k] Y_k with respect to (x, y, z) of the formulas above.
__device__ __forceinline__ void sh_grad(int deg, float x, float y, float z, const float g[16],
                                        float &gx, float &gy, float &gz) {
  gx = gy = gz = 0.f;
  if (deg < 1) return;
  gy += kSH1 * g[1]; gz += kSH1 * g[2]; gx += kSH1 * g[3];
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  gx += kSH2a * (y * g[4] + z * g[7]) + kSH2c * 2.f * x * g[8];
  gy += kSH2a * (x * g[4] + z * g[5]) - kSH2c * 2.f * y * g[8];
  gz += kSH2a * (y * g[5] + x * g[7]) + kSH2b * 6.f * z * g[6];
  if (deg < 3) return;
  // Y9 = a y (3x^2 - y^2)
  gx += kSH3a * 6.f * x * y * g[9];
  gy += kSH3a * (3.f * xx - 3.f * yy) * g[9];
  // Y10 = b x y z
  gx += kSH3b * y * z * g[10]; gy += kSH3b * x * z * g[10]; gz += kSH3b * x * y * g[10];
  // Y11 = c y (5 z^2 - 1)
  gy += kSH3c * (5.f * zz - 1.f) * g[11]; gz += kSH3c * 10.f * y * z * g[11];
  // Y12 = d z (5 z^2 - 3) = d (5 z^3 - 3 z)
  gz += kSH3d * (15.f * zz - 3.f) * g[12];
  // Y13 = c x (5 z^2 - 1)
  gx += kSH3c * (5.f * zz - 1.f) * g[13]; gz += kSH3c * 10.f * x * z * g[13];
  // Y14 = e z (x^2 - y^2)
  gx += kSH3e * 2.f * x * z * g[14]; gy -= kSH3e * 2.f * y * z * g[14];
  gz += kSH3e * (xx - yy) * g[14];
  // Y15 = a x (x^2 - 3 y^2)
  gx += kSH3a * (3.f * xx - 3.f * yy) * g[15]; gy -= kSH3a * 6.f * x * y * g[15];
}

// The time- and camera-independent part of a Gaussian's forward: the 4D frame from the two
// quaternions and the scales, and Eq. 1's conditional factors (N with Sigma_xyz|t = N N^T,
// w with mu(t) = mu_xyz + w (t - mu_t) / |m_t|, Sigma_t = |m_t|^2) and sigmoid(o).
__device__ __forceinline__ void gauss_cond(float4 ls, float4 ql, float4 qr, float o,
                                           GaussState &g, float &inv_nt) {
  quat_unit(ql, g.qn_l, g.inv_l);
  quat_unit(qr, g.qn_r, g.inv_r);
  left_mat(g.qn_l, g.Lm);
  right_mat(g.qn_r, g.Rm);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc = fmaf(g.Lm[i * 4 + k], g.Rm[k * 4 + j], acc);
      g.R[i * 4 + j] = acc;
    }
  g.s[0] = expf(ls.x); g.s[1] = expf(ls.y); g.s[2] = expf(ls.z); g.s[3] = expf(ls.w);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) g.M[i * 4 + j] = g.R[i * 4 + j] * g.s[j];
  // Eq. 1 / Eq. 3
  g.nt2 = g.M[12] * g.M[12] + g.M[13] * g.M[13] + g.M[14] * g.M[14] + g.M[15] * g.M[15];
  g.nt = sqrtf(g.nt2);
  inv_nt = 1.f / g.nt;
#pragma unroll
  for (int m = 0; m < 4; ++m) g.mh[m] = g.M[12 + m] * inv_nt;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    g.w[j] = g.M[j * 4 + 0] * g.mh[0] + g.M[j * 4 + 1] * g.mh[1] + g.M[j * 4 + 2] * g.mh[2] +
             g.M[j * 4 + 3] * g.mh[3];
#pragma unroll
    for (int m = 0; m < 4; ++m) g.N[j * 4 + m] = g.M[j * 4 + m] - g.w[j] * g.mh[m];
  }
  g.sig = 1.f / (1.f + expf(-o));
}

// The per-(t, camera) part of the forward, from the conditional factors (g.N, g.w, g.nt2,
// g.sig and inv_nt): temporal weight, conditional mean, view transform, EWA projection, up
// to the cull tests. Returns the decision flags (kFlag*); a Gaussian that fails a test stops
// there. cull = false keeps a Gaussian whose a = sigmoid(o) p(t) is below 1/255 (it can
// reach alpha >= 1/255 nowhere, so the image is the same; its flag bit stays clear).
__device__ __forceinline__ uint8_t gauss_forward_tail(const DevCam &cam, float t, float4 mean,
                                                      float inv_nt, GaussState &g,
                                                      bool cull = true) {
  uint8_t flags = kFlagMask;
  g.dt = t - mean.w;
  g.p = expf(-0.5f * g.dt * g.dt / g.nt2);
  g.a = g.sig * g.p;
  if (g.a >= kAlphaMin)
    flags |= kFlagTemporal;
  else if (cull)
    return flags;
  const float k = g.dt * inv_nt;
  g.mu3[0] = mean.x + g.w[0] * k;
  g.mu3[1] = mean.y + g.w[1] * k;
  g.mu3[2] = mean.z + g.w[2] * k;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    g.xc[r] = cam.R[r * 3 + 0] * g.mu3[0] + cam.R[r * 3 + 1] * g.mu3[1] +
              cam.R[r * 3 + 2] * g.mu3[2] + cam.tv[r];
  if (!(g.xc[2] > cam.znear)) return flags;
  flags |= kFlagNear;
  g.iz = 1.f / g.xc[2];
  g.xr = g.xc[0] * g.iz;
  g.yr = g.xc[1] * g.iz;
  g.clx = (g.xr < -cam.limx) || (g.xr > cam.limx);
  g.cly = (g.yr < -cam.limy) || (g.yr > cam.limy);
  g.xz = fminf(fmaxf(g.xr, -cam.limx), cam.limx);
  g.yz = fminf(fmaxf(g.yr, -cam.limy), cam.limy);
  const float ax = cam.fx * g.iz, ay = cam.fy * g.iz;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    g.T2[j] = ax * (cam.R[j] - g.xz * cam.R[6 + j]);
    g.T2[3 + j] = ay * (cam.R[3 + j] - g.yz * cam.R[6 + j]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int m = 0; m < 4; ++m)
      g.P[r * 4 + m] = g.T2[r * 3 + 0] * g.N[m] + g.T2[r * 3 + 1] * g.N[4 + m] +
                       g.T2[r * 3 + 2] * g.N[8 + m];
  const float p00 = g.P[0] * g.P[0] + g.P[1] * g.P[1] + g.P[2] * g.P[2] + g.P[3] * g.P[3];
  const float p11 = g.P[4] * g.P[4] + g.P[5] * g.P[5] + g.P[6] * g.P[6] + g.P[7] * g.P[7];
  g.c01 = g.P[0] * g.P[4] + g.P[1] * g.P[5] + g.P[2] * g.P[6] + g.P[3] * g.P[7];
  g.c00 = p00 + kDilation;
  g.c11 = p11 + kDilation;
  float minors = 0.f;
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int n = m + 1; n < 4; ++n) {
      float d = g.P[m] * g.P[4 + n] - g.P[n] * g.P[4 + m];
      minors = fmaf(d, d, minors);
    }
  g.det = minors + kDilation * (p00 + p11) + kDilation * kDilation;
  if (!(g.det > 0.f)) return flags;
  flags |= kFlagDet;
  return flags;
}

// Forward of one Gaussian up to the cull tests (both parts). Returns the decision flags
// (kFlag*). The state is filled as far as the Gaussian got.
__device__ __forceinline__ uint8_t gauss_forward(const DevCam &cam, float t, float4 mean,
                                                 float4 ls, float4 ql, float4 qr, float o,
                                                 GaussState &g, bool cull = true) {
  float inv_nt;
  gauss_cond(ls, ql, qr, o, g, inv_nt);
  return gauss_forward_tail(cam, t, mean, inv_nt, g, cull);
}

// The conditional factors of gauss_cond as stored per Gaussian for the batched path
// (5 x float4): N (12), w (3), inv_nt, nt2, sigmoid(o), 2 unused.
constexpr int kCond4 = 5;
__device__ __forceinline__ void cond_store(const GaussState &g, float inv_nt, float4 *dst) {
  dst[0] = make_float4(g.N[0], g.N[1], g.N[2], g.N[3]);
  dst[1] = make_float4(g.N[4], g.N[5], g.N[6], g.N[7]);
  dst[2] = make_float4(g.N[8], g.N[9], g.N[10], g.N[11]);
  dst[3] = make_float4(g.w[0], g.w[1], g.w[2], inv_nt);
  dst[4] = make_float4(g.nt2, g.sig, 0.f, 0.f);
}
__device__ __forceinline__ void cond_load(const float4 *__restrict__ src, GaussState &g,
                                          float &inv_nt) {
  const float4 a = __ldg(&src[0]), b = __ldg(&src[1]), c = __ldg(&src[2]),
               d = __ldg(&src[3]), e = __ldg(&src[4]);
  g.N[0] = a.x; g.N[1] = a.y; g.N[2] = a.z; g.N[3] = a.w;
  g.N[4] = b.x; g.N[5] = b.y; g.N[6] = b.z; g.N[7] = b.w;
  g.N[8] = c.x; g.N[9] = c.y; g.N[10] = c.z; g.N[11] = c.w;
  g.w[0] = d.x; g.w[1] = d.y; g.w[2] = d.z; inv_nt = d.w;
  g.nt2 = e.x; g.sig = e.y;
}

// Colour of a Gaussian that reached the projection (state has mu3), from its SH coefficients
// coef(k, c) (band-major k = 0 .. (deg+1)^2 - 1, channel c): the view direction from the
// camera centre to the conditional mean, the real SH basis, max(0, sum + 0.5).
template <typename Coef>
__device__ __forceinline__ void gauss_colour_from(const DevCam &cam, int deg, GaussState &g,
                                                  float rgb[3], Coef &&coef) {
  float d0 = g.mu3[0] - cam.eye[0], d1 = g.mu3[1] - cam.eye[1], d2 = g.mu3[2] - cam.eye[2];
  g.dlen = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  const float il = 1.f / g.dlen;
  g.dn[0] = d0 * il; g.dn[1] = d1 * il; g.dn[2] = d2 * il;
  float Y[16];
  sh_eval(deg, g.dn[0], g.dn[1], g.dn[2], Y);
  const int K = (deg + 1) * (deg + 1);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float acc = 0.5f;
    for (int k = 0; k < K; ++k) acc = fmaf(Y[k], coef(k, c), acc);
    g.raw[c] = acc;
    rgb[c] = fmaxf(acc, 0.f);
  }
}

// The colour with the coefficients read from sh [K][3][n], or, with kVQ, the DC plane from sh
// and bands k >= 1 from cb[code[i]][k - 1][c] (vector-quantised SH). kVQ is a template
// parameter so that the full-coefficient kernels carry none of the codebook path.
template <bool kVQ = false>
__device__ __forceinline__ void gauss_colour(const DevCam &cam, const float *__restrict__ sh,
                                             const float *__restrict__ cb,
                                             const uint16_t *__restrict__ code, int deg,
                                             int64_t n, int64_t i, GaussState &g,
                                             float rgb[3]) {
  const int K = (deg + 1) * (deg + 1);
  const float *row = kVQ ? cb + (size_t)__ldg(&code[i]) * (size_t)(K - 1) * 3 : nullptr;
  gauss_colour_from(cam, deg, g, rgb, [&](int k, int c) {
    return (kVQ && k > 0) ? __ldg(&row[(k - 1) * 3 + c])
                          : __ldg(&sh[((int64_t)k * 3 + c) * n + i]);
  });
}

// Gradients of one Gaussian's parameters from the gradients of its 2D record:
// gu, gv (image position), gA, gB, gC (conic), ga (opacity x temporal weight), grgb.
// Adds into the output gradient arrays at index i. The state must hold a full forward.
struct GaussGrad {
  float mean[4], ls[4], ql[4], qr[4], o;
};

__device__ __forceinline__ void gauss_backward(const DevCam &cam, const float *__restrict__ sh,
                                               int deg, int64_t n, int64_t i,
                                               const GaussState &g, float gu, float gv,
                                               float gA, float gB, float gC, float ga,
                                               const float grgb[3], GaussGrad &out,
                                               float *g_sh) {
  // ---- colour (SH) ----
  float graw[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) graw[c] = g.raw[c] > 0.f ? grgb[c] : 0.f;
  float Y[16];
  sh_eval(deg, g.dn[0], g.dn[1], g.dn[2], Y);
  const int K = (deg + 1) * (deg + 1);
  float gk[16];
  for (int k = 0; k < K; ++k) {
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t idx = ((int64_t)k * 3 + c) * n + i;
      acc = fmaf(__ldg(&sh[idx]), graw[c], acc);
      if (g_sh) g_sh[idx] += Y[k] * graw[c];
    }
    gk[k] = acc;
  }
  float gmu3[3] = {0.f, 0.f, 0.f};
  if (deg > 0) {
    float gdx, gdy, gdz;
    sh_grad(deg, g.dn[0], g.dn[1], g.dn[2], gk, gdx, gdy, gdz);
    const float dot = gdx * g.dn[0] + gdy * g.dn[1] + gdz * g.dn[2];
    const float il = 1.f / g.dlen;
    gmu3[0] = (gdx - g.dn[0] * dot) * il;
    gmu3[1] = (gdy - g.dn[1] * dot) * il;
    gmu3[2] = (gdz - g.dn[2] * dot) * il;
  }
  // ---- conic -> 2D covariance ----
  const float idet = 1.f / g.det;
  const float idet2 = idet * idet;
  const float gdet = -(gA * g.c11 - gB * g.c01 + gC * g.c00) * idet2;
  const float gc00 = gC * idet + gdet * g.c11;
  const float gc11 = gA * idet + gdet * g.c00;
  const float gc01 = -gB * idet - 2.f * gdet * g.c01;
  // ---- 2D covariance -> P = T N ----
  float gP[8];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    gP[m] = 2.f * gc00 * g.P[m] + gc01 * g.P[4 + m];
    gP[4 + m] = 2.f * gc11 * g.P[4 + m] + gc01 * g.P[m];
  }
  // ---- P -> T (2x3) and N (3x4) ----
  float gT[6], gN[12];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      gT[r * 3 + j] = gP[r * 4 + 0] * g.N[j * 4 + 0] + gP[r * 4 + 1] * g.N[j * 4 + 1] +
                      gP[r * 4 + 2] * g.N[j * 4 + 2] + gP[r * 4 + 3] * g.N[j * 4 + 3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int m = 0; m < 4; ++m) gN[j * 4 + m] = g.T2[j] * gP[m] + g.T2[3 + j] * gP[4 + m];
  // ---- T = J R_view -> iz, clamped ratios ----
  float giz = 0.f, gxz = 0.f, gyz = 0.f;
  {
    float s0 = 0.f, s1 = 0.f, r0 = 0.f, r1 = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      s0 += gT[j] * (cam.R[j] - g.xz * cam.R[6 + j]);
      s1 += gT[3 + j] * (cam.R[3 + j] - g.yz * cam.R[6 + j]);
      r0 += gT[j] * cam.R[6 + j];
      r1 += gT[3 + j] * cam.R[6 + j];
    }
    giz = cam.fx * s0 + cam.fy * s1;
    gxz = -cam.fx * g.iz * r0;
    gyz = -cam.fy * g.iz * r1;
  }
  float gxr = cam.fx * gu + (g.clx ? 0.f : gxz);
  float gyr = cam.fy * gv + (g.cly ? 0.f : gyz);
  // xr = x iz, yr = y iz, iz = 1/z
  float gxc[3];
  gxc[0] = gxr * g.iz;
  gxc[1] = gyr * g.iz;
  giz += gxr * g.xc[0] + gyr * g.xc[1];
  gxc[2] = -giz * g.iz * g.iz;
  // xc = R_view mu3 + tv
#pragma unroll
  for (int j = 0; j < 3; ++j)
    gmu3[j] += cam.R[j] * gxc[0] + cam.R[3 + j] * gxc[1] + cam.R[6 + j] * gxc[2];
  // ---- slice: mu3 = mu_xyz + w dt / nt; p = exp(-dt^2 / (2 nt2)); a = sig p ----
  const float inv_nt = 1.f / g.nt;
  float gw[3], gdt = 0.f, gnt = 0.f, gnt2 = 0.f;
  const float gmw = gmu3[0] * g.w[0] + gmu3[1] * g.w[1] + gmu3[2] * g.w[2];
#pragma unroll
  for (int j = 0; j < 3; ++j) gw[j] = gmu3[j] * g.dt * inv_nt;
  gdt += gmw * inv_nt;
  gnt -= gmw * g.dt * inv_nt * inv_nt;
  const float gsig = ga * g.p;
  const float gp = ga * g.sig;
  out.o = gsig * g.sig * (1.f - g.sig);
  gdt += gp * g.p * (-g.dt / g.nt2);
  gnt2 += gp * g.p * 0.5f * g.dt * g.dt / (g.nt2 * g.nt2);
  // ---- N = M_x - w m^T, w = M_x m^ ----
  float gM[16], gmh[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) acc += gN[j * 4 + m] * g.mh[m];
    gw[j] -= acc;
  }
#pragma unroll
  for (int m = 0; m < 4; ++m)
    gmh[m] -= gN[m] * g.w[0] + gN[4 + m] * g.w[1] + gN[8 + m] * g.w[2];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      gM[j * 4 + m] = gN[j * 4 + m] + gw[j] * g.mh[m];
      gmh[m] += g.M[j * 4 + m] * gw[j];
    }
  // m^ = m_t / nt, nt = |m_t|, nt2 = |m_t|^2
  {
    const float dot = gmh[0] * g.mh[0] + gmh[1] * g.mh[1] + gmh[2] * g.mh[2] + gmh[3] * g.mh[3];
#pragma unroll
    for (int m = 0; m < 4; ++m)
      gM[12 + m] = (gmh[m] - g.mh[m] * dot) * inv_nt + gnt * g.mh[m] + 2.f * gnt2 * g.M[12 + m];
  }
  // ---- M = R diag(s), s = exp(ls) ----
  float gR[16];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      gR[j * 4 + m] = gM[j * 4 + m] * g.s[m];
      acc += gM[j * 4 + m] * g.R[j * 4 + m];
    }
    out.ls[m] = acc * g.s[m];
  }
  // ---- R = Lm Rm ----
  float gL[16], gRr[16];
#pragma unroll
  for (int i2 = 0; i2 < 4; ++i2)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        a1 += gR[i2 * 4 + j] * g.Rm[k * 4 + j];   // gL = gR Rm^T
        a2 += g.Lm[j * 4 + i2] * gR[j * 4 + k];   // gRm = Lm^T gR
      }
      gL[i2 * 4 + k] = a1;
      gRr[i2 * 4 + k] = a2;
    }
  float gql[4], gqr[4];
  gql[0] = gL[0] + gL[5] + gL[10] + gL[15];
  gql[1] = -gL[1] + gL[4] - gL[11] + gL[14];
  gql[2] = -gL[2] + gL[7] + gL[8] - gL[13];
  gql[3] = -gL[3] - gL[6] + gL[9] + gL[12];
  gqr[0] = gRr[0] + gRr[5] + gRr[10] + gRr[15];
  gqr[1] = -gRr[1] + gRr[4] + gRr[11] - gRr[14];
  gqr[2] = -gRr[2] - gRr[7] + gRr[8] + gRr[13];
  gqr[3] = -gRr[3] + gRr[6] - gRr[9] + gRr[12];
  {
    const float dl = gql[0] * g.qn_l[0] + gql[1] * g.qn_l[1] + gql[2] * g.qn_l[2] + gql[3] * g.qn_l[3];
    const float dr = gqr[0] * g.qn_r[0] + gqr[1] * g.qn_r[1] + gqr[2] * g.qn_r[2] + gqr[3] * g.qn_r[3];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      out.ql[m] = (gql[m] - g.qn_l[m] * dl) * g.inv_l;
      out.qr[m] = (gqr[m] - g.qn_r[m] * dr) * g.inv_r;
    }
  }
  out.mean[0] = gmu3[0];
  out.mean[1] = gmu3[1];
  out.mean[2] = gmu3[2];
  out.mean[3] = -gdt;
}

}  // namespace fdgs
