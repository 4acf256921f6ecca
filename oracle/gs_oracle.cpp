/*
 * gs_oracle.cpp -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, single-threaded CPU restatement of what the hot path of On-the-Fly GS computes
 * on every Local & Semi-Global iteration: the differentiable 3D Gaussian Splatting rasterizer
 * that the paper builds on (Sec. III, Eq. 1 and Eq. 2, with "all other settings" of the
 * original 3DGS per Sec. V-A), the L1 + D-SSIM part of the loss (Eq. 10), the analytic gradients
 * of all of it, and the Adam step.  Only tests/, the package's smoke check and bench.py's CPU
 * baseline may load this library; the product never does.  It shares no source, header, table
 * or helper with the CUDA path.
 *
 * Every routine is templated on the scalar type.  The float instantiation takes every
 * threshold decision (alpha cutoff, termination, clamps) in fp32, the precision of the kernels;
 * the double instantiation serves finite differences and closed forms.  No blocking, fusion or
 * reordering: per Gaussian, per tile, per pixel, in the natural order.
 *
 * Parameter layout (one Gaussian = 59 scalars, component-major with a row stride):
 *   params[c * stride + i];  c = 0..2 mean xyz, 3..5 log-scale, 6..9 quaternion (w,x,y,z),
 *   10 opacity logit, 11 + 3k + ch SH coefficient k (0..15) of colour channel ch (0..2).
 * Camera (double[16]): R row-major world->camera (0..8), t (9..11), fx, fy, cx, cy (12..15);
 *   x_cam = R x_world + t, u = fx x/z + cx, v = fy y/z + cy; pixel (px, py) is sampled at the
 *   continuous image point (px, py).
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

constexpr int kParams = 59;
constexpr double kNear = 0.2;        // cull at z <= 0.2 (3DGS near plane)
constexpr double kDilation = 0.3;    // added to the 2D covariance diagonal (3DGS low-pass filter)
constexpr double kFovClamp = 1.3;    // x/z, y/z clamped to 1.3 x half-FOV tangent when forming J
constexpr double kAlphaMax = 0.99;   // alpha clamp
constexpr double kTransMin = 1e-4;   // stop before a Gaussian that takes T below this

template <class T>
struct Cam {
  T R[9], t[3], fx, fy, cx, cy;
  int W, H;
};

template <class T>
Cam<T> load_cam(const double* c, int W, int H) {
  Cam<T> k;
  for (int i = 0; i < 9; ++i) k.R[i] = (T)c[i];
  for (int i = 0; i < 3; ++i) k.t[i] = (T)c[9 + i];
  k.fx = (T)c[12];
  k.fy = (T)c[13];
  k.cx = (T)c[14];
  k.cy = (T)c[15];
  k.W = W;
  k.H = H;
  return k;
}

// Real spherical harmonics up to degree 3 with the Condon-Shortley phase, in the basis ordering
// of 3DGS.  The constants are the orthonormalisation factors sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
// written out as closed forms and evaluated here, not tabulated.
template <class T>
struct SH {
  T c0, c1, c2a, c2b, c2c, c3a, c3b, c3c, c3d, c3e;
  SH() {
    const double pi = 3.14159265358979323846;
    c0 = (T)(0.5 * std::sqrt(1.0 / pi));
    c1 = (T)std::sqrt(3.0 / (4.0 * pi));
    c2a = (T)(0.5 * std::sqrt(15.0 / pi));
    c2b = (T)(0.25 * std::sqrt(5.0 / pi));
    c2c = (T)(0.25 * std::sqrt(15.0 / pi));
    c3a = (T)(0.25 * std::sqrt(35.0 / (2.0 * pi)));
    c3b = (T)(0.5 * std::sqrt(105.0 / pi));
    c3c = (T)(0.25 * std::sqrt(21.0 / (2.0 * pi)));
    c3d = (T)(0.25 * std::sqrt(7.0 / pi));
    c3e = (T)(0.25 * std::sqrt(105.0 / pi));
  }
  void eval(T x, T y, T z, T Y[16]) const {
    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c2b * (2 * z * z - x * x - y * y);
    Y[7] = -c2a * x * z;
    Y[8] = c2c * (x * x - y * y);
    Y[9] = -c3a * y * (3 * x * x - y * y);
    Y[10] = c3b * x * y * z;
    Y[11] = -c3c * y * (4 * z * z - x * x - y * y);
    Y[12] = c3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
    Y[13] = -c3c * x * (4 * z * z - x * x - y * y);
    Y[14] = c3e * z * (x * x - y * y);
    Y[15] = -c3a * x * (x * x - 3 * y * y);
  }
  // dY[k][0..2] = partial derivatives of Y_k with respect to x, y, z (x, y, z independent).
  void grad(T x, T y, T z, T dY[16][3]) const {
    for (int k = 0; k < 16; ++k) dY[k][0] = dY[k][1] = dY[k][2] = 0;
    dY[1][1] = -c1;
    dY[2][2] = c1;
    dY[3][0] = -c1;
    dY[4][0] = c2a * y;
    dY[4][1] = c2a * x;
    dY[5][1] = -c2a * z;
    dY[5][2] = -c2a * y;
    dY[6][0] = -2 * c2b * x;
    dY[6][1] = -2 * c2b * y;
    dY[6][2] = 4 * c2b * z;
    dY[7][0] = -c2a * z;
    dY[7][2] = -c2a * x;
    dY[8][0] = 2 * c2c * x;
    dY[8][1] = -2 * c2c * y;
    dY[9][0] = -6 * c3a * x * y;
    dY[9][1] = -c3a * (3 * x * x - 3 * y * y);
    dY[10][0] = c3b * y * z;
    dY[10][1] = c3b * x * z;
    dY[10][2] = c3b * x * y;
    dY[11][0] = 2 * c3c * x * y;
    dY[11][1] = -c3c * (4 * z * z - x * x - 3 * y * y);
    dY[11][2] = -8 * c3c * y * z;
    dY[12][0] = -6 * c3d * x * z;
    dY[12][1] = -6 * c3d * y * z;
    dY[12][2] = c3d * (6 * z * z - 3 * x * x - 3 * y * y);
    dY[13][0] = -c3c * (4 * z * z - 3 * x * x - y * y);
    dY[13][1] = 2 * c3c * x * y;
    dY[13][2] = -8 * c3c * x * z;
    dY[14][0] = 2 * c3e * x * z;
    dY[14][1] = -2 * c3e * y * z;
    dY[14][2] = c3e * (x * x - y * y);
    dY[15][0] = -c3a * (3 * x * x - 3 * y * y);
    dY[15][1] = 6 * c3a * x * y;
  }
};

// Tile rectangle of a projected Gaussian (3DGS rule): tiles [x0, x1) x [y0, y1) covered by the
// square of half-side r around (u, v), clamped to the grid.  Evaluated in the scalar type T.
template <class T>
void rect_of(T u, T v, int r, int tw, int th, int gx, int gy, int rect[4], T* margin) {
  using std::fabs;
  using std::floor;
  using std::round;
  const T rr = (T)r;
  T q[4];
  q[0] = (u - rr) / (T)tw;
  q[1] = (v - rr) / (T)th;
  q[2] = ((u + rr) + (T)(tw - 1)) / (T)tw;
  q[3] = ((v + rr) + (T)(th - 1)) / (T)th;
  const int lim[4] = {gx, gy, gx, gy};
  for (int k = 0; k < 4; ++k) {
    T f = floor(q[k]);
    long long iv = (long long)f;
    if (iv < 0) iv = 0;
    if (iv > lim[k]) iv = lim[k];
    rect[k] = (int)iv;
    if (margin) {
      T d = fabs(q[k] - round(q[k]));
      if (d < *margin) *margin = d;
    }
  }
}

// Everything the forward projection of one Gaussian into one view computes; the backward
// recomputes it rather than storing it.
template <class T>
struct Proj {
  bool visible = false;
  T p[3];
  T q[4], qn[4], qlen;
  T Rq[9], s[3], M[9], Sig[9];
  bool xin, yin;
  T txz, tyz;
  T J[6], Tm[6];
  T cov[3];
  T det;
  T conic[3];
  T u, v;
  T lam, rf;
  int radius = 0;
  int rect[4] = {0, 0, 0, 0};
  T dvec[3], dlen, dir[3];
  T Y[16];
  T raw[3], rgb[3];
  uint8_t clampbits = 0;
  T opacity;
  T margin;
};

template <class T>
Proj<T> project_one(const T* params, int64_t i, int64_t stride, const Cam<T>& cam, int tw, int th,
                    const SH<T>& sh) {
  using std::ceil;
  using std::exp;
  using std::fabs;
  using std::isfinite;
  using std::round;
  using std::sqrt;
  Proj<T> f;
  auto P = [&](int c) { return params[(int64_t)c * stride + i]; };
  const T mu[3] = {P(0), P(1), P(2)};
  for (int r = 0; r < 3; ++r)
    f.p[r] = cam.R[3 * r + 0] * mu[0] + cam.R[3 * r + 1] * mu[1] + cam.R[3 * r + 2] * mu[2] + cam.t[r];
  f.margin = std::numeric_limits<T>::infinity();
  if (!(f.p[2] > (T)kNear)) return f;  // behind the near plane (also rejects NaN)

  // Eq. 1: Sigma = R S S^T R^T from the (normalised) quaternion and exp(log-scale).
  for (int k = 0; k < 4; ++k) f.q[k] = P(6 + k);
  f.qlen = sqrt(f.q[0] * f.q[0] + f.q[1] * f.q[1] + f.q[2] * f.q[2] + f.q[3] * f.q[3]);
  if (!(f.qlen > 0)) return f;
  for (int k = 0; k < 4; ++k) f.qn[k] = f.q[k] / f.qlen;
  const T w = f.qn[0], x = f.qn[1], y = f.qn[2], z = f.qn[3];
  f.Rq[0] = 1 - 2 * (y * y + z * z);
  f.Rq[1] = 2 * (x * y - w * z);
  f.Rq[2] = 2 * (x * z + w * y);
  f.Rq[3] = 2 * (x * y + w * z);
  f.Rq[4] = 1 - 2 * (x * x + z * z);
  f.Rq[5] = 2 * (y * z - w * x);
  f.Rq[6] = 2 * (x * z - w * y);
  f.Rq[7] = 2 * (y * z + w * x);
  f.Rq[8] = 1 - 2 * (x * x + y * y);
  for (int k = 0; k < 3; ++k) f.s[k] = exp(P(3 + k));
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) f.M[3 * r + c] = f.Rq[3 * r + c] * f.s[c];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      T acc = 0;
      for (int k = 0; k < 3; ++k) acc += f.M[3 * r + k] * f.M[3 * c + k];
      f.Sig[3 * r + c] = acc;
    }

  // EWA: Sigma_2D = J W Sigma W^T J^T + 0.3 I with J the Jacobian of the pinhole map at the
  // (FOV-clamped) camera-space mean.
  const T pz = f.p[2];
  const T limx = (T)kFovClamp * ((T)cam.W / (2 * cam.fx));
  const T limy = (T)kFovClamp * ((T)cam.H / (2 * cam.fy));
  const T xz = f.p[0] / pz, yz = f.p[1] / pz;
  f.xin = (xz >= -limx) && (xz <= limx);
  f.yin = (yz >= -limy) && (yz <= limy);
  f.txz = std::min(limx, std::max(-limx, xz));
  f.tyz = std::min(limy, std::max(-limy, yz));
  f.J[0] = cam.fx / pz;
  f.J[1] = 0;
  f.J[2] = -cam.fx * f.txz / pz;
  f.J[3] = 0;
  f.J[4] = cam.fy / pz;
  f.J[5] = -cam.fy * f.tyz / pz;
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) {
      T acc = 0;
      for (int k = 0; k < 3; ++k) acc += f.J[3 * r + k] * cam.R[3 * k + c];
      f.Tm[3 * r + c] = acc;
    }
  T S2[4];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      T acc = 0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) acc += f.Tm[3 * r + a] * f.Sig[3 * a + b] * f.Tm[3 * c + b];
      S2[2 * r + c] = acc;
    }
  f.cov[0] = S2[0] + (T)kDilation;
  f.cov[1] = S2[1];
  f.cov[2] = S2[3] + (T)kDilation;
  f.det = f.cov[0] * f.cov[2] - f.cov[1] * f.cov[1];
  if (!(f.det > 0)) return f;
  f.conic[0] = f.cov[2] / f.det;
  f.conic[1] = -f.cov[1] / f.det;
  f.conic[2] = f.cov[0] / f.det;
  f.u = cam.fx * f.p[0] / pz + cam.cx;
  f.v = cam.fy * f.p[1] / pz + cam.cy;
  const T mid = (T)0.5 * (f.cov[0] + f.cov[2]);
  f.lam = mid + sqrt(std::max((T)0.1, mid * mid - f.det));
  f.rf = 3 * sqrt(f.lam);
  f.radius = (int)ceil(f.rf);
  {
    T d = fabs(f.rf - round(f.rf));
    if (d < f.margin) f.margin = d;
  }
  const int gx = (cam.W + tw - 1) / tw, gy = (cam.H + th - 1) / th;
  rect_of<T>(f.u, f.v, f.radius, tw, th, gx, gy, f.rect, &f.margin);
  if ((f.rect[2] - f.rect[0]) * (f.rect[3] - f.rect[1]) == 0) return f;
  if (!(isfinite(f.u) && isfinite(f.v) && isfinite(f.conic[0]) &&
        isfinite(f.conic[1]) && isfinite(f.conic[2])))
    return f;

  // Colour from degree-3 SH at the view direction (mean minus camera centre), + 0.5, >= 0.
  T campos[3];
  for (int c = 0; c < 3; ++c)
    campos[c] = -(cam.R[0 * 3 + c] * cam.t[0] + cam.R[1 * 3 + c] * cam.t[1] + cam.R[2 * 3 + c] * cam.t[2]);
  for (int c = 0; c < 3; ++c) f.dvec[c] = mu[c] - campos[c];
  f.dlen = sqrt(f.dvec[0] * f.dvec[0] + f.dvec[1] * f.dvec[1] + f.dvec[2] * f.dvec[2]);
  for (int c = 0; c < 3; ++c) f.dir[c] = f.dvec[c] / f.dlen;
  sh.eval(f.dir[0], f.dir[1], f.dir[2], f.Y);
  f.clampbits = 0;
  for (int ch = 0; ch < 3; ++ch) {
    T acc = 0;
    for (int k = 0; k < 16; ++k) acc += f.Y[k] * P(11 + 3 * k + ch);
    f.raw[ch] = acc + (T)0.5;
    if (f.raw[ch] < 0) f.clampbits |= (uint8_t)(1u << ch);
    f.rgb[ch] = std::max((T)0, f.raw[ch]);
  }
  f.opacity = (T)1 / ((T)1 + exp(-P(10)));
  f.visible = true;
  return f;
}

template <class T>
void project(const T* params, int64_t n, int64_t stride, const double* camd, int W, int H, int tw,
             int th, T* mean2d, T* depth, T* conic, T* opacity, T* rgb, int32_t* radius,
             int32_t* rect, uint8_t* clampbits, T* margin) {
  const Cam<T> cam = load_cam<T>(camd, W, H);
  const SH<T> sh;
  for (int64_t i = 0; i < n; ++i) {
    Proj<T> f = project_one<T>(params, i, stride, cam, tw, th, sh);
    if (margin) margin[i] = f.margin;
    if (!f.visible) {
      radius[i] = 0;
      for (int k = 0; k < 4; ++k) rect[4 * i + k] = 0;
      mean2d[2 * i] = mean2d[2 * i + 1] = 0;
      depth[i] = f.p[2];
      conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0;
      opacity[i] = 0;
      rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0;
      clampbits[i] = 0;
      continue;
    }
    radius[i] = f.radius;
    for (int k = 0; k < 4; ++k) rect[4 * i + k] = f.rect[k];
    mean2d[2 * i] = f.u;
    mean2d[2 * i + 1] = f.v;
    depth[i] = f.p[2];
    for (int k = 0; k < 3; ++k) conic[3 * i + k] = f.conic[k];
    opacity[i] = f.opacity;
    for (int k = 0; k < 3; ++k) rgb[3 * i + k] = f.rgb[k];
    clampbits[i] = f.clampbits;
  }
}

uint32_t float_bits(float f) {
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return b;
}

// Duplication into (tile, depth) keys, the sort and the per-tile ranges, by brute force: every
// (Gaussian, tile) pair of every view is enumerated with the rect rule and the pairs are put in
// the canonical order (global tile, fp32 depth bits, record index).
int64_t build_lists(int V, int64_t n, const int* Ws, const int* Hs, int tw, int th,
                    const float* mean2d, const int32_t* radius, const float* depth, int64_t cap,
                    uint64_t* keys, uint32_t* vals, uint32_t* ranges) {
  struct Inst {
    uint64_t key;
    uint32_t val;
  };
  std::vector<Inst> inst;
  std::vector<int64_t> base(V + 1, 0);
  for (int v = 0; v < V; ++v) {
    const int gx = (Ws[v] + tw - 1) / tw, gy = (Hs[v] + th - 1) / th;
    base[v + 1] = base[v] + (int64_t)gx * gy;
  }
  for (int v = 0; v < V; ++v) {
    const int gx = (Ws[v] + tw - 1) / tw, gy = (Hs[v] + th - 1) / th;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t rec = (int64_t)v * n + i;
      if (radius[rec] <= 0) continue;
      int rect[4];
      rect_of<float>(mean2d[2 * rec], mean2d[2 * rec + 1], radius[rec], tw, th, gx, gy, rect, nullptr);
      for (int ty = rect[1]; ty < rect[3]; ++ty)
        for (int tx = rect[0]; tx < rect[2]; ++tx) {
          const uint64_t tile = (uint64_t)(base[v] + (int64_t)ty * gx + tx);
          inst.push_back({(tile << 32) | float_bits(depth[rec]), (uint32_t)rec});
        }
    }
  }
  std::sort(inst.begin(), inst.end(), [](const Inst& a, const Inst& b) {
    if (a.key != b.key) return a.key < b.key;
    return a.val < b.val;
  });
  const int64_t m = (int64_t)inst.size();
  for (int64_t t = 0; t < base[V]; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
  for (int64_t k = 0; k < m; ++k) {
    const uint64_t tile = inst[k].key >> 32;
    if (k == 0 || (inst[k - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)k;
    if (k == m - 1 || (inst[k + 1].key >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(k + 1);
    if (k < cap) {
      keys[k] = inst[k].key;
      vals[k] = inst[k].val;
    }
  }
  return m;
}

// Eq. 2, per pixel, front to back over the pixel's tile list (3DGS blending rule with its alpha
// cutoff 1/255, clamp 0.99 and the early stop before T would fall below 1e-4).
template <class T>
struct PixelWalk {
  struct Contrib {
    uint32_t rec;
    T alpha, Tb, G, dx, dy;
    bool clamped;
  };
  std::vector<Contrib> contrib;
  T trans, C[3];
  uint32_t last, neval, gp;
  T margin;
};

template <class T>
void walk_pixel(int px, int py, uint32_t start, uint32_t end, const uint32_t* vals,
                const T* mean2d, const T* conic, const T* opacity, const T* rgb, PixelWalk<T>& w,
                bool keep) {
  const T one255 = (T)1 / (T)255;
  const T amax = (T)kAlphaMax, tmin = (T)kTransMin;
  w.contrib.clear();
  w.trans = 1;
  w.C[0] = w.C[1] = w.C[2] = 0;
  w.last = 0;
  w.gp = 0;
  w.margin = std::numeric_limits<T>::infinity();
  const uint32_t L = end - start;
  w.neval = L;
  for (uint32_t j = 0; j < L; ++j) {
    const uint32_t rec = vals[start + j];
    const T dx = mean2d[2 * rec] - (T)px;
    const T dy = mean2d[2 * rec + 1] - (T)py;
    const T a = conic[3 * rec], b = conic[3 * rec + 1], c = conic[3 * rec + 2];
    const T power = (T)(-0.5) * (a * dx * dx + c * dy * dy) - b * dx * dy;
    if (power > 0) continue;
    const T G = std::exp(power);
    const T oG = opacity[rec] * G;
    const T alpha = std::min(amax, oG);
    w.margin = std::min(w.margin, std::fabs(alpha - one255) / one255);
    if (alpha < one255) continue;
    const T testT = w.trans * (1 - alpha);
    w.margin = std::min(w.margin, std::fabs(testT - tmin) / tmin);
    if (testT < tmin) {
      w.neval = j + 1;
      break;
    }
    if (keep) w.contrib.push_back({rec, alpha, w.trans, G, dx, dy, oG > amax});
    for (int ch = 0; ch < 3; ++ch) w.C[ch] += rgb[3 * rec + ch] * alpha * w.trans;
    w.trans = testT;
    w.last = j + 1;
    w.gp += 1;
  }
}

template <class T>
void blend_forward(int W, int H, int tw, int th, int64_t tile_base, const uint32_t* ranges,
                   const uint32_t* vals, const T* mean2d, const T* conic, const T* opacity,
                   const T* rgb, const T* bg, T* img, T* Tout, uint32_t* last, uint32_t* neval,
                   uint32_t* gp, T* margin) {
  const int gx = (W + tw - 1) / tw;
  PixelWalk<T> w;
  const int64_t HW = (int64_t)W * H;
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      const int64_t tile = tile_base + (int64_t)(py / th) * gx + px / tw;
      walk_pixel<T>(px, py, ranges[2 * tile], ranges[2 * tile + 1], vals, mean2d, conic, opacity, rgb,
                    w, false);
      const int64_t pix = (int64_t)py * W + px;
      for (int ch = 0; ch < 3; ++ch) img[ch * HW + pix] = w.C[ch] + w.trans * bg[ch];
      Tout[pix] = w.trans;
      last[pix] = w.last;
      neval[pix] = w.neval;
      gp[pix] = w.gp;
      if (margin) margin[pix] = w.margin;
    }
}

// Gradient of Eq. 2 in the natural per-pixel order: the forward walk keeps every contributor
// with its exact transmittance, then the contributors are visited back to front while the colour
// behind them (including the background term) is accumulated.  The clamps and cutoffs act as
// masks.  grad2d per record: d mean2d (2), d conic (a, b, c), d opacity, d rgb (3).  load_w
// (nullable) is dL/dG_p per pixel for the load-balancing term of Eq. 9-10; G_p is a count, and its
// derivative is taken through the soft count of blend_soft_count below (the sum of the alphas).
//
// With kMagnitude the same walk accumulates, instead of each gradient, the sum of the absolute
// values of every elementary product that enters it (|dL/dC| |c| T, |a dx| + |b dy| for the mean,
// ...), and terms[rec] counts the (pixel, contributor) terms summed into the record.  The colour
// behind a contributor enters at the scale of the pixel's whole colour (sum of |c| alpha T over
// all contributors plus |bg| T): it equals the pixel colour minus the colour in front, and a
// front-to-back evaluation obtains it as that difference, whose rounding is relative to the
// operands.  That is the scale of the componentwise
// rounding-error bound of the sum (Higham, "Accuracy and Stability of Numerical Algorithms", Sec.
// 4.2: |fl(sum) - sum| <= gamma_k sum |x_i| for k terms): a parity check uses it for the entries
// whose terms cancel.
template <class T, bool kMagnitude>
void blend_backward_impl(int W, int H, int tw, int th, int64_t tile_base, const uint32_t* ranges,
                         const uint32_t* vals, const T* mean2d, const T* conic, const T* opacity,
                         const T* rgb, const T* bg, const T* dimg, const T* load_w, T* grad2d, uint32_t* terms) {
  const int gx = (W + tw - 1) / tw;
  PixelWalk<T> w;
  const int64_t HW = (int64_t)W * H;
  auto mag = [](T x) { return kMagnitude ? std::fabs(x) : x; };
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      const int64_t tile = tile_base + (int64_t)(py / th) * gx + px / tw;
      walk_pixel<T>(px, py, ranges[2 * tile], ranges[2 * tile + 1], vals, mean2d, conic, opacity, rgb,
                    w, true);
      const int64_t pix = (int64_t)py * W + px;
      T dC[3], S[3];
      for (int ch = 0; ch < 3; ++ch) {
        dC[ch] = mag(dimg[ch * HW + pix]);
        S[ch] = mag(bg[ch]) * w.trans;
      }
      if (kMagnitude)  // the scale of the colour behind any contributor: the pixel's whole colour
        for (const auto& e : w.contrib)
          for (int ch = 0; ch < 3; ++ch) S[ch] += std::fabs(rgb[3 * e.rec + ch]) * e.alpha * e.Tb;
      for (int k = (int)w.contrib.size() - 1; k >= 0; --k) {
        const auto& e = w.contrib[k];
        T* g = grad2d + 9 * (int64_t)e.rec;
        if (terms) terms[e.rec] += 1;
        const T wgt = e.alpha * e.Tb;
        T dalpha = 0;
        for (int ch = 0; ch < 3; ++ch) {
          const T c = mag(rgb[3 * e.rec + ch]);
          g[6 + ch] += wgt * dC[ch];
          if (kMagnitude) {
            dalpha += dC[ch] * (c * e.Tb + S[ch] / (1 - e.alpha));
          } else {
            dalpha += dC[ch] * (c * e.Tb - S[ch] / (1 - e.alpha));
            S[ch] += c * wgt;
          }
        }
        // Eq. 9 through the soft count: dL_load/dG_p (load_w) x d alpha / d alpha
        if (load_w) dalpha += mag(load_w[pix]);
        if (e.clamped) continue;
        const T a = conic[3 * e.rec], b = conic[3 * e.rec + 1], c = conic[3 * e.rec + 2];
        g[5] += dalpha * e.G;
        const T dpower = dalpha * e.alpha;
        if (kMagnitude) {
          g[0] += dpower * (std::fabs(a * e.dx) + std::fabs(b * e.dy));
          g[1] += dpower * (std::fabs(c * e.dy) + std::fabs(b * e.dx));
        } else {
          g[0] += dpower * (-(a * e.dx + b * e.dy));
          g[1] += dpower * (-(c * e.dy + b * e.dx));
        }
        g[2] += mag(dpower * ((T)(-0.5) * e.dx * e.dx));
        g[3] += mag(dpower * (-(e.dx * e.dy)));
        g[4] += mag(dpower * ((T)(-0.5) * e.dy * e.dy));
      }
    }
}

template <class T>
void blend_backward(int W, int H, int tw, int th, int64_t tile_base, const uint32_t* ranges,
                    const uint32_t* vals, const T* mean2d, const T* conic, const T* opacity,
                    const T* rgb, const T* bg, const T* dimg, const T* load_w, T* grad2d) {
  blend_backward_impl<T, false>(W, H, tw, th, tile_base, ranges, vals, mean2d, conic, opacity, rgb, bg,
                                dimg, load_w, grad2d, nullptr);
}

// The soft count of Eq. 9's G_p: per pixel, the sum of the alphas of the Gaussians it blends (each
// Gaussian counted by how much it is associated with the pixel).  Its value is not used by the
// loss (L_load takes the count itself); its derivative is the one the backward gives the count.
template <class T>
void blend_soft_count(int W, int H, int tw, int th, int64_t tile_base, const uint32_t* ranges,
                      const uint32_t* vals, const T* mean2d, const T* conic, const T* opacity, const T* rgb,
                      T* soft) {
  const int gx = (W + tw - 1) / tw;
  PixelWalk<T> w;
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      const int64_t tile = tile_base + (int64_t)(py / th) * gx + px / tw;
      walk_pixel<T>(px, py, ranges[2 * tile], ranges[2 * tile + 1], vals, mean2d, conic, opacity, rgb, w, true);
      T acc = 0;
      for (const auto& e : w.contrib) acc += e.alpha;
      soft[(int64_t)py * W + px] = acc;
    }
}

// Chain rule of one visible Gaussian in one view: its 2D gradient g2 (9 values) back to its 59
// parameters, accumulated through G(c); P(c) reads its parameters.
template <class T, class PF, class GF>
void chain_one(const Proj<T>& f, const Cam<T>& cam, const SH<T>& sh, const T* g2, PF P, GF G) {
  T dmu[3] = {0, 0, 0};
  T dp[3] = {0, 0, 0};

  // opacity = sigmoid(logit)
  G(10) += g2[5] * f.opacity * (1 - f.opacity);

  // colour -> SH coefficients and view direction
  T ddir[3] = {0, 0, 0};
  T dY[16][3];
  sh.grad(f.dir[0], f.dir[1], f.dir[2], dY);
  for (int ch = 0; ch < 3; ++ch) {
    if (f.clampbits & (1u << ch)) continue;
    const T dcol = g2[6 + ch];
    for (int k = 0; k < 16; ++k) {
      G(11 + 3 * k + ch) += f.Y[k] * dcol;
      for (int a = 0; a < 3; ++a) ddir[a] += dY[k][a] * P(11 + 3 * k + ch) * dcol;
    }
  }
  const T dd = f.dir[0] * ddir[0] + f.dir[1] * ddir[1] + f.dir[2] * ddir[2];
  for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - f.dir[a] * dd) / f.dlen;

  // conic = inverse of the dilated covariance (a', b', c'), written out per entry
  const T A = f.cov[0], B = f.cov[1], C = f.cov[2], det = f.det, det2 = det * det;
  const T dA = g2[2], dB = g2[3], dC = g2[4];
  const T da = dA * (-C * C / det2) + dB * (B * C / det2) + dC * (1 / det - A * C / det2);
  const T db = dA * (2 * B * C / det2) + dB * (-1 / det - 2 * B * B / det2) + dC * (2 * A * B / det2);
  const T dc = dA * (1 / det - A * C / det2) + dB * (A * B / det2) + dC * (-A * A / det2);

  // (a, b, c) = entries of Tm Sigma Tm^T, Tm = J R_cam (2 x 3)
  T dSig[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      dSig[3 * r + c] = da * f.Tm[r] * f.Tm[c] + db * f.Tm[r] * f.Tm[3 + c] + dc * f.Tm[3 + r] * f.Tm[3 + c];
  T dTm[6] = {0, 0, 0, 0, 0, 0};
  for (int r = 0; r < 3; ++r) {
    T s00 = 0, s01 = 0, s10 = 0, s11 = 0;
    for (int k = 0; k < 3; ++k) {
      const T sym = f.Sig[3 * r + k] + f.Sig[3 * k + r];
      s00 += sym * f.Tm[k];
      s11 += sym * f.Tm[3 + k];
      s01 += f.Sig[3 * r + k] * f.Tm[3 + k];
      s10 += f.Sig[3 * k + r] * f.Tm[k];
    }
    dTm[r] += da * s00 + db * s01;
    dTm[3 + r] += dc * s11 + db * s10;
  }
  T dJ[6];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) {
      T acc = 0;
      for (int k = 0; k < 3; ++k) acc += dTm[3 * r + k] * cam.R[3 * c + k];
      dJ[3 * r + c] = acc;
    }
  const T x = f.p[0], y = f.p[1], z = f.p[2], z2 = z * z, z3 = z2 * z;
  dp[2] += dJ[0] * (-cam.fx / z2) + dJ[4] * (-cam.fy / z2);
  if (f.xin) {
    dp[0] += dJ[2] * (-cam.fx / z2);
    dp[2] += dJ[2] * (2 * cam.fx * x / z3);
  } else {
    dp[2] += dJ[2] * (cam.fx * f.txz / z2);
  }
  if (f.yin) {
    dp[1] += dJ[5] * (-cam.fy / z2);
    dp[2] += dJ[5] * (2 * cam.fy * y / z3);
  } else {
    dp[2] += dJ[5] * (cam.fy * f.tyz / z2);
  }
  // mean2d = (fx x/z + cx, fy y/z + cy)
  dp[0] += g2[0] * cam.fx / z;
  dp[2] += g2[0] * (-cam.fx * x / z2);
  dp[1] += g2[1] * cam.fy / z;
  dp[2] += g2[1] * (-cam.fy * y / z2);
  for (int a = 0; a < 3; ++a)
    dmu[a] += cam.R[0 * 3 + a] * dp[0] + cam.R[1 * 3 + a] * dp[1] + cam.R[2 * 3 + a] * dp[2];
  for (int a = 0; a < 3; ++a) G(a) += dmu[a];

  // Sigma = M M^T, M = R_q diag(s)
  T dM[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      T acc = 0;
      for (int k = 0; k < 3; ++k) acc += (dSig[3 * r + k] + dSig[3 * k + r]) * f.M[3 * k + c];
      dM[3 * r + c] = acc;
    }
  T dRq[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) dRq[3 * r + c] = dM[3 * r + c] * f.s[c];
  for (int c = 0; c < 3; ++c) {
    T ds = 0;
    for (int r = 0; r < 3; ++r) ds += dM[3 * r + c] * f.Rq[3 * r + c];
    G(3 + c) += ds * f.s[c];
  }
  const T w = f.qn[0], qx = f.qn[1], qy = f.qn[2], qz = f.qn[3];
  T dqn[4];
  dqn[0] = dRq[1] * (-2 * qz) + dRq[2] * (2 * qy) + dRq[3] * (2 * qz) + dRq[5] * (-2 * qx) +
           dRq[6] * (-2 * qy) + dRq[7] * (2 * qx);
  dqn[1] = dRq[1] * (2 * qy) + dRq[2] * (2 * qz) + dRq[3] * (2 * qy) + dRq[4] * (-4 * qx) +
           dRq[5] * (-2 * w) + dRq[6] * (2 * qz) + dRq[7] * (2 * w) + dRq[8] * (-4 * qx);
  dqn[2] = dRq[0] * (-4 * qy) + dRq[1] * (2 * qx) + dRq[2] * (2 * w) + dRq[3] * (2 * qx) +
           dRq[5] * (2 * qz) + dRq[6] * (-2 * w) + dRq[7] * (2 * qz) + dRq[8] * (-4 * qy);
  dqn[3] = dRq[0] * (-4 * qz) + dRq[1] * (-2 * w) + dRq[2] * (2 * qx) + dRq[3] * (2 * w) +
           dRq[4] * (-4 * qz) + dRq[5] * (2 * qy) + dRq[6] * (2 * qx) + dRq[7] * (2 * qy);
  const T qd = f.qn[0] * dqn[0] + f.qn[1] * dqn[1] + f.qn[2] * dqn[2] + f.qn[3] * dqn[3];
  for (int k = 0; k < 4; ++k) G(6 + k) += (dqn[k] - f.qn[k] * qd) / f.qlen;
}

// Chain rule from the per-view 2D quantities back to the 59 parameters of each Gaussian,
// accumulated into grads (component-major, same stride as params).
template <class T>
void project_backward(const T* params, int64_t n, int64_t stride, const double* camd, int W, int H,
                      int tw, int th, const T* grad2d, T* grads) {
  const Cam<T> cam = load_cam<T>(camd, W, H);
  const SH<T> sh;
  for (int64_t i = 0; i < n; ++i) {
    const Proj<T> f = project_one<T>(params, i, stride, cam, tw, th, sh);
    if (!f.visible) continue;
    auto G = [&](int c) -> T& { return grads[(int64_t)c * stride + i]; };
    auto P = [&](int c) { return params[(int64_t)c * stride + i]; };
    chain_one<T>(f, cam, sh, grad2d + 9 * i, P, G);
  }
}

// L = (1 - lambda) mean|X - Y| + lambda (1 - mean SSIM(X, Y)), means over 3 H W.  SSIM uses an
// 11 x 11 Gaussian window (sigma 1.5, normalised), zero padding, "same" size, C1 = 0.01^2,
// C2 = 0.03^2, per channel.  X is the render, Y the target; the gradient is with respect to X.
// Every window sum is evaluated directly in 2D.
template <class T>
double loss(int W, int H, const T* X, const T* Y, double lambda, T* dX, double grad_scale,
            double* out_l1, double* out_ssim) {
  const int R = 5;
  double w1[11], wsum = 0;
  for (int k = -R; k <= R; ++k) {
    w1[k + R] = std::exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
    wsum += w1[k + R];
  }
  T w2[11][11];
  for (int a = 0; a < 11; ++a)
    for (int b = 0; b < 11; ++b) w2[a][b] = (T)((w1[a] / wsum) * (w1[b] / wsum));
  const T C1 = (T)(0.01 * 0.01), C2 = (T)(0.03 * 0.03);
  const int64_t HW = (int64_t)W * H;
  const double count = 3.0 * (double)HW;
  double l1 = 0, ssim = 0;
  std::vector<T> dmu(HW), dxx(HW), dxy(HW);
  const T gS = (T)(-lambda / count * grad_scale);
  const T gL1 = (T)((1.0 - lambda) / count * grad_scale);
  for (int ch = 0; ch < 3; ++ch) {
    const T* x = X + ch * HW;
    const T* y = Y + ch * HW;
    for (int py = 0; py < H; ++py)
      for (int px = 0; px < W; ++px) {
        T mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
        for (int a = -R; a <= R; ++a)
          for (int b = -R; b <= R; ++b) {
            const int qy = py + a, qx = px + b;
            if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;
            const T wt = w2[a + R][b + R];
            const T xv = x[(int64_t)qy * W + qx], yv = y[(int64_t)qy * W + qx];
            mx += wt * xv;
            my += wt * yv;
            exx += wt * xv * xv;
            eyy += wt * yv * yv;
            exy += wt * xv * yv;
          }
        const T N1 = 2 * mx * my + C1, N2 = 2 * (exy - mx * my) + C2;
        const T D1 = mx * mx + my * my + C1, D2 = (exx - mx * mx) + (eyy - my * my) + C2;
        const T N = N1 * N2, D = D1 * D2;
        const T S = N / D;
        ssim += (double)S;
        const int64_t p = (int64_t)py * W + px;
        const T dN_dmx = 2 * my * N2 + N1 * (-2 * my);
        const T dD_dmx = 2 * mx * D2 + D1 * (-2 * mx);
        dmu[p] = (dN_dmx * D - N * dD_dmx) / (D * D);
        dxx[p] = -N * D1 / (D * D);
        dxy[p] = 2 * N1 / D;
        const T diff = x[p] - y[p];
        l1 += std::fabs((double)diff);
      }
    if (dX) {
      T* dx = dX + ch * HW;
      for (int qy = 0; qy < H; ++qy)
        for (int qx = 0; qx < W; ++qx) {
          const int64_t q = (int64_t)qy * W + qx;
          const T diff = x[q] - y[q];
          T g = diff > 0 ? gL1 : (diff < 0 ? -gL1 : (T)0);
          T acc = 0;
          for (int a = -R; a <= R; ++a)
            for (int b = -R; b <= R; ++b) {
              const int py = qy + a, px = qx + b;
              if (py < 0 || py >= H || px < 0 || px >= W) continue;
              const int64_t p = (int64_t)py * W + px;
              acc += w2[a + R][b + R] * (dmu[p] + 2 * x[q] * dxx[p] + y[q] * dxy[p]);
            }
          dx[q] = g + gS * acc;
        }
    }
  }
  l1 /= count;
  ssim /= count;
  if (out_l1) *out_l1 = l1;
  if (out_ssim) *out_ssim = ssim;
  return (1.0 - lambda) * l1 + lambda * (1.0 - ssim);
}

// Adam (bias-corrected, torch.optim.Adam's update) with one learning rate per parameter group:
// 0 means (c 0..2), 1 log-scales (3..5), 2 quaternions (6..9), 3 opacity (10), 4 SH DC
// (11..13), 5 SH rest (14..58).
int group_of(int c) {
  if (c < 3) return 0;
  if (c < 6) return 1;
  if (c < 10) return 2;
  if (c < 11) return 3;
  if (c < 14) return 4;
  return 5;
}

template <class T>
void adam(T* params, const T* grads, T* m, T* v, int64_t n, int64_t stride, const double* lr,
          double b1, double b2, double eps, int64_t step) {
  const double bc1 = 1.0 - std::pow(b1, (double)step);
  const double bc2 = 1.0 - std::pow(b2, (double)step);
  for (int c = 0; c < kParams; ++c) {
    const T step_size = (T)(lr[group_of(c)] / bc1);
    const T bc2s = (T)std::sqrt(bc2);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t k = (int64_t)c * stride + i;
      const T g = grads[k];
      m[k] = (T)b1 * m[k] + (T)(1.0 - b1) * g;
      v[k] = (T)b2 * v[k] + (T)(1.0 - b2) * g * g;
      params[k] -= step_size * m[k] / (std::sqrt(v[k]) / bc2s + (T)eps);
    }
  }
}

template <class T>
void sh_eval_export(const T* dirs, int64_t n, T* out) {
  const SH<T> sh;
  for (int64_t i = 0; i < n; ++i) sh.eval(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], out + 16 * i);
}

// The rounding scale of the projection and its chain rule: a value carried with the sum of the
// magnitudes of the products it was built from (a sum or difference adds the magnitudes, a product
// multiplies them, a quotient divides by the divisor's magnitude; an input, and the result of a
// square root or an exponential, is its own magnitude).  Evaluating the projection and the chain
// in this type gives, per parameter gradient, the sum of |products| of the componentwise
// rounding-error bound (Higham, "Accuracy and Stability of Numerical Algorithms", Sec. 3.1-3.3):
// |fl(g) - g| <= gamma_k x magnitude for an evaluation of depth k.  Branch decisions (clamps,
// visibility, the tile rectangle) are taken on the values.
struct Mag {
  double v, m;
  Mag(double x = 0.0) : v(x), m(std::fabs(x)) {}
  Mag(double x, double mm) : v(x), m(mm) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
  explicit operator long long() const { return (long long)v; }
};
inline Mag operator+(Mag a, Mag b) { return Mag(a.v + b.v, a.m + b.m); }
inline Mag operator-(Mag a, Mag b) { return Mag(a.v - b.v, a.m + b.m); }
inline Mag operator-(Mag a) { return Mag(-a.v, a.m); }
inline Mag operator*(Mag a, Mag b) { return Mag(a.v * b.v, a.m * b.m); }
inline Mag operator/(Mag a, Mag b) { return Mag(a.v / b.v, a.m / std::fabs(b.v)); }
inline Mag& operator+=(Mag& a, Mag b) { return a = a + b; }
inline bool operator<(Mag a, Mag b) { return a.v < b.v; }
inline bool operator>(Mag a, Mag b) { return a.v > b.v; }
inline bool operator<=(Mag a, Mag b) { return a.v <= b.v; }
inline bool operator>=(Mag a, Mag b) { return a.v >= b.v; }
inline Mag sqrt(Mag a) { return Mag(std::sqrt(a.v)); }
inline Mag exp(Mag a) { return Mag(std::exp(a.v)); }
inline Mag floor(Mag a) { return Mag(std::floor(a.v)); }
inline Mag ceil(Mag a) { return Mag(std::ceil(a.v)); }
inline Mag round(Mag a) { return Mag(std::round(a.v)); }
inline Mag fabs(Mag a) { return Mag(std::fabs(a.v), a.m); }
inline bool isfinite(Mag a) { return std::isfinite(a.v); }

// Magnitudes of the products that make up each parameter gradient of the projection backward
// (accumulated into grads_mag, component-major like params), for fp64 parameters and 2D gradients.
void project_backward_magnitude(const double* params, int64_t n, int64_t stride, const double* camd, int W,
                                int H, int tw, int th, const double* grad2d, double* grads_mag) {
  const Cam<Mag> cam = load_cam<Mag>(camd, W, H);
  const SH<Mag> sh;
  for (int64_t i = 0; i < n; ++i) {
    Mag pm[kParams], g2[9], acc[kParams];
    for (int c = 0; c < kParams; ++c) pm[c] = Mag(params[(int64_t)c * stride + i]);
    const Proj<Mag> f = project_one<Mag>(pm, 0, 1, cam, tw, th, sh);
    if (!f.visible) continue;
    for (int k = 0; k < 9; ++k) g2[k] = Mag(grad2d[9 * i + k]);
    auto G = [&](int c) -> Mag& { return acc[c]; };
    auto P = [&](int c) { return pm[c]; };
    chain_one<Mag>(f, cam, sh, g2, P, G);
    for (int c = 0; c < kParams; ++c) grads_mag[(int64_t)c * stride + i] += acc[c].m;
  }
}

}  // namespace

extern "C" {

#define ORC_EXPORT __attribute__((visibility("default")))

#define ORC_INSTANTIATE(T, SUF)                                                                    \
  ORC_EXPORT void orc_project_##SUF(const T* params, int64_t n, int64_t stride, const double* cam,  \
                                    int W, int H, int tw, int th, T* mean2d, T* depth, T* conic,    \
                                    T* opacity, T* rgb, int32_t* radius, int32_t* rect,             \
                                    uint8_t* clampbits, T* margin) {                                 \
    project<T>(params, n, stride, cam, W, H, tw, th, mean2d, depth, conic, opacity, rgb, radius,   \
               rect, clampbits, margin);                                                           \
  }                                                                                                \
  ORC_EXPORT void orc_blend_forward_##SUF(int W, int H, int tw, int th, int64_t tile_base,          \
                                          const uint32_t* ranges, const uint32_t* vals,             \
                                          const T* mean2d, const T* conic, const T* opacity,        \
                                          const T* rgb, const T* bg, T* img, T* Tout,               \
                                          uint32_t* last, uint32_t* neval, uint32_t* gp,            \
                                          T* margin) {                                              \
    blend_forward<T>(W, H, tw, th, tile_base, ranges, vals, mean2d, conic, opacity, rgb, bg, img,  \
                     Tout, last, neval, gp, margin);                                               \
  }                                                                                                \
  ORC_EXPORT void orc_blend_backward_##SUF(int W, int H, int tw, int th, int64_t tile_base,         \
                                           const uint32_t* ranges, const uint32_t* vals,            \
                                           const T* mean2d, const T* conic, const T* opacity,       \
                                           const T* rgb, const T* bg, const T* dimg,                \
                                           const T* load_w, T* grad2d) {                            \
    blend_backward<T>(W, H, tw, th, tile_base, ranges, vals, mean2d, conic, opacity, rgb, bg,      \
                      dimg, load_w, grad2d);                                                       \
  }                                                                                                \
  ORC_EXPORT void orc_blend_soft_count_##SUF(int W, int H, int tw, int th, int64_t tile_base,       \
                                             const uint32_t* ranges, const uint32_t* vals,          \
                                             const T* mean2d, const T* conic, const T* opacity,     \
                                             const T* rgb, T* soft) {                               \
    blend_soft_count<T>(W, H, tw, th, tile_base, ranges, vals, mean2d, conic, opacity, rgb, soft); \
  }                                                                                                \
  ORC_EXPORT void orc_blend_backward_magnitude_##SUF(                                             \
      int W, int H, int tw, int th, int64_t tile_base, const uint32_t* ranges, const uint32_t* vals, \
      const T* mean2d, const T* conic, const T* opacity, const T* rgb, const T* bg, const T* dimg,   \
      const T* load_w, T* grad2d_mag, uint32_t* terms) {                                           \
    blend_backward_impl<T, true>(W, H, tw, th, tile_base, ranges, vals, mean2d, conic, opacity,    \
                                 rgb, bg, dimg, load_w, grad2d_mag, terms);                       \
  }                                                                                                \
  ORC_EXPORT void orc_project_backward_##SUF(const T* params, int64_t n, int64_t stride,            \
                                             const double* cam, int W, int H, int tw, int th,       \
                                             const T* grad2d, T* grads) {                           \
    project_backward<T>(params, n, stride, cam, W, H, tw, th, grad2d, grads);                      \
  }                                                                                                \
  ORC_EXPORT double orc_loss_##SUF(int W, int H, const T* X, const T* Y, double lambda, T* dX,      \
                                   double grad_scale, double* out_l1, double* out_ssim) {           \
    return loss<T>(W, H, X, Y, lambda, dX, grad_scale, out_l1, out_ssim);                          \
  }                                                                                                \
  ORC_EXPORT void orc_adam_##SUF(T* params, const T* grads, T* m, T* v, int64_t n, int64_t stride,  \
                                 const double* lr, double b1, double b2, double eps,                \
                                 int64_t step) {                                                    \
    adam<T>(params, grads, m, v, n, stride, lr, b1, b2, eps, step);                                \
  }                                                                                                \
  ORC_EXPORT void orc_sh_eval_##SUF(const T* dirs, int64_t n, T* out) {                             \
    sh_eval_export<T>(dirs, n, out);                                                               \
  }

ORC_INSTANTIATE(float, f32)
ORC_INSTANTIATE(double, f64)

ORC_EXPORT void orc_project_backward_magnitude(const double* params, int64_t n, int64_t stride,
                                               const double* cam, int W, int H, int tw, int th,
                                               const double* grad2d, double* grads_mag) {
  project_backward_magnitude(params, n, stride, cam, W, H, tw, th, grad2d, grads_mag);
}

ORC_EXPORT int64_t orc_build_lists(int V, int64_t n, const int* Ws, const int* Hs, int tw, int th,
                                   const float* mean2d, const int32_t* radius, const float* depth,
                                   int64_t cap, uint64_t* keys, uint32_t* vals, uint32_t* ranges) {
  return build_lists(V, n, Ws, Hs, tw, th, mean2d, radius, depth, cap, keys, vals, ranges);
}

}  // extern "C"
