// Differentiable camera (arXiv 1611.01652, section 3.4: the inverted pendulum observed by a camera).
// A pinhole ray tracer over textured objects carried by the bodies (oriented boxes, spheres,
// planes), batched over instances: four pixels per thread. The pixel (i, j) ray leaves the camera
// centre C along d = R_c^T (P ((j + 1/2) - W/2) / f, P ((i + 1/2) - H/2) / f, P), so t = 1 is the
// projection plane at distance P; every object is intersected in its own frame (boxes: slab
// test; spheres: |o + t d| = r; planes: the frame's z = 0), and of the hits at t >= 1 (in front
// of the projection plane) the nearest is kept. Texture coordinates come from the hit point in
// the object's frame (box: the entry face, u = (x_a / h_a + 1) / 2, v = (x_b / h_b + 1) / 2 with
// a = k+1, b = k+2 mod 3 for face axis k; sphere: u = atan2(y, x) / (2 pi) + 1/2,
// v = acos(z / r) / pi; plane: u = frac(x / (2 h_0) + 1/2), v = frac(y / (2 h_1) + 1/2)) and the
// colour is the bilinear interpolation of the object's texture (texel centres at
// ((c + 1/2) / Wt, (r + 1/2) / Ht), clamped at the edges), so the frame has non-zero derivatives
// with respect to the state and the texels. Reverse mode keeps the forward pass's discrete
// choices (object, face, texels, texture period) and differentiates the rest.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <string>

#include "../../include/dp.h"

namespace {

constexpr int kMaxObj = DP_CAMERA_MAX_OBJECTS;
constexpr int kThreads = 256, kPixPerThread = 4, kChunk = kThreads * kPixPerThread;

struct CamArgs {
  int W, H, B, nb, n_obj, th, tw;
  int cull;  // screen rectangles per object (DP_CAMERA_NO_CULL turns them off, for comparison)
  float f, plane;
  float pf, invW;  // plane / f and 1 / W (per-pixel arithmetic without divisions)
  float C[3], Rc[9];
  int body[kMaxObj], tex[kMaxObj], kind[kMaxObj];
  float cen[kMaxObj][3], half[kMaxObj][3];
};

struct Hit {
  int obj, k;          // k: the entry face's axis (boxes); -1 sphere, -2 plane
  float t;
  float ol[3], dl[3];  // ray origin and direction in the hit object's frame
};

// Frame of one box for one instance: R (box to world), centre c_w, and the camera centre in the
// box frame o = R^T (C - c_w) (the same for every pixel); when the frames are staged per block,
// also the object's screen rectangle (rect: j_lo, j_hi, i_lo, i_hi): pixels outside it cannot hit
// the object.
struct BoxFrame {
  float R[9], cw[3], o[3];
  float rect[4];
  // staged frames: the ray direction in the object's frame is affine in the pixel's camera
  // coordinates (x, y) = (P/f (j + 1/2 - W/2), P/f (i + 1/2 - H/2)): dl = x e[0..2] + y e[3..5] +
  // e[6..8], with e the object's R^T times the camera's first two rows and P times its third
  float e[9];
};

__device__ __forceinline__ float pick3(const float (&v)[3], int k) { return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]); }

__device__ __forceinline__ void box_frame(const CamArgs& A, const float* __restrict__ state, int inst, int o, BoxFrame& F) {
  const int b = A.body[o];
  float p[3];
  if (b >= 0) {
    const float* x = state + ((size_t)inst * A.nb + b) * 18;
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = __ldg(x + k);
#pragma unroll
    for (int k = 0; k < 9; ++k) F.R[k] = __ldg(x + 3 + k);
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) F.R[k] = (k % 4 == 0) ? 1.f : 0.f;
    p[0] = p[1] = p[2] = 0.f;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) F.cw[r] = p[r] + F.R[3 * r] * A.cen[o][0] + F.R[3 * r + 1] * A.cen[o][1] + F.R[3 * r + 2] * A.cen[o][2];
#pragma unroll
  for (int k = 0; k < 3; ++k) F.o[k] = F.R[k] * (A.C[0] - F.cw[0]) + F.R[3 + k] * (A.C[1] - F.cw[1]) + F.R[6 + k] * (A.C[2] - F.cw[2]);
}

// Screen rectangle of object o (frame F): a point q in camera coordinates (q = R_c (x - C)) lies on
// the ray of pixel (i, j) when j + 1/2 = f q_0 / q_2 + W / 2 and i + 1/2 = f q_1 / q_2 + H / 2, at
// the ray parameter t = q_2 / P. When every corner of the object's box (a sphere's: the cube
// around it) is in front of the camera (q_2 > 0), the object's image is the convex hull of the
// projected corners, so a pixel outside their bounding rectangle (widened by one pixel for
// rounding) cannot hit it; when every corner lies before the projection plane (q_2 < P), no ray
// hits it at t >= 1. Otherwise (a corner behind the camera, or a plane) every pixel tests it.
__device__ __forceinline__ void screen_rect(const CamArgs& A, int o, BoxFrame& F) {
  F.rect[0] = F.rect[2] = -INFINITY;
  F.rect[1] = F.rect[3] = INFINITY;
  if (!A.cull || A.kind[o] == DP_OBJ_PLANE) return;
  const float h0 = A.half[o][0];
  const float h1 = A.kind[o] == DP_OBJ_SPHERE ? h0 : A.half[o][1];
  const float h2 = A.kind[o] == DP_OBJ_SPHERE ? h0 : A.half[o][2];
  float jlo = INFINITY, jhi = -INFINITY, ilo = INFINITY, ihi = -INFINITY, zmax = -INFINITY;
  for (int c = 0; c < 8; ++c) {
    const float l[3] = {c & 1 ? h0 : -h0, c & 2 ? h1 : -h1, c & 4 ? h2 : -h2};
    float w[3], q[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) w[r] = F.cw[r] + F.R[3 * r] * l[0] + F.R[3 * r + 1] * l[1] + F.R[3 * r + 2] * l[2] - A.C[r];
#pragma unroll
    for (int k = 0; k < 3; ++k) q[k] = A.Rc[3 * k] * w[0] + A.Rc[3 * k + 1] * w[1] + A.Rc[3 * k + 2] * w[2];
    if (!(q[2] > 0.f)) return;  // a corner behind the camera: no bound
    zmax = fmaxf(zmax, q[2]);
    const float jc = A.f * q[0] / q[2] + 0.5f * (float)A.W - 0.5f, ic = A.f * q[1] / q[2] + 0.5f * (float)A.H - 0.5f;
    jlo = fminf(jlo, jc);
    jhi = fmaxf(jhi, jc);
    ilo = fminf(ilo, ic);
    ihi = fmaxf(ihi, ic);
  }
  if (zmax < A.plane) {  // wholly before the projection plane
    F.rect[0] = F.rect[2] = INFINITY;
    F.rect[1] = F.rect[3] = -INFINITY;
    return;
  }
  F.rect[0] = jlo - 1.f;
  F.rect[1] = jhi + 1.f;
  F.rect[2] = ilo - 1.f;
  F.rect[3] = ihi + 1.f;
}

// Work split: a block takes kChunk consecutive pixels of the batch, kPixPerThread per thread
// (pixel first + threadIdx.x + r kThreads). When W * H is a multiple of kChunk every block lies in
// one instance and its box frames are computed once into shared memory; otherwise each thread
// computes its own (see `trace`).
__device__ __forceinline__ bool stage_frames(const CamArgs& A, const float* __restrict__ state, BoxFrame* sf, int& inst0,
                                             int& pix0) {
  const int npix = A.W * A.H;
  const int chunks = npix / kChunk;
  const bool uniform = npix % kChunk == 0;
  inst0 = uniform ? (int)(blockIdx.x / chunks) : 0;
  pix0 = uniform ? (int)(blockIdx.x % chunks) * kChunk : 0;
  if (uniform)
    for (int o = threadIdx.x; o < A.n_obj; o += blockDim.x) {
      box_frame(A, state, inst0, o, sf[o]);
      screen_rect(A, o, sf[o]);
      BoxFrame& F = sf[o];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        F.e[k] = F.R[k] * A.Rc[0] + F.R[3 + k] * A.Rc[1] + F.R[6 + k] * A.Rc[2];
        F.e[3 + k] = F.R[k] * A.Rc[3] + F.R[3 + k] * A.Rc[4] + F.R[6 + k] * A.Rc[5];
        F.e[6 + k] = A.plane * (F.R[k] * A.Rc[6] + F.R[3 + k] * A.Rc[7] + F.R[6 + k] * A.Rc[8]);
      }
    }
  __syncthreads();
  return uniform;
}
// Instance and pixel of the r-th pixel of this thread.
__device__ __forceinline__ bool pixel_of(const CamArgs& A, bool uniform, int inst0, int pix0, int r, int& inst, int& pix) {
  const int npix = A.W * A.H;
  if (uniform) {
    inst = inst0;
    pix = pix0 + (int)threadIdx.x + r * kThreads;
    return true;
  }
  const long long idx = (long long)blockIdx.x * kChunk + threadIdx.x + (long long)r * kThreads;
  if (idx >= (long long)npix * A.B) return false;
  inst = (int)(idx / npix);
  pix = (int)(idx - (long long)inst * npix);
  return true;
}

// Row i and column j of pixel pix: the float quotient (pix < W H < 2^24, exact in float; the
// product with the rounded 1/W is within one row), moved by one row when rounding put it across a
// row boundary, so the result is exact.
__device__ __forceinline__ void pixel_ij(const CamArgs& A, int pix, int& i, int& j) {
  int q = (int)(((float)pix + 0.5f) * A.invW);
  int r = pix - q * A.W;
  if (r < 0) {
    --q;
    r += A.W;
  } else if (r >= A.W) {
    ++q;
    r -= A.W;
  }
  i = q;
  j = r;
}

__device__ __forceinline__ void ray_dir(const CamArgs& A, int i, int j, float d[3]) {
  const float dc0 = A.plane * (((float)j + 0.5f) - 0.5f * (float)A.W) / A.f;
  const float dc1 = A.plane * (((float)i + 0.5f) - 0.5f * (float)A.H) / A.f;
  const float dc2 = A.plane;
#pragma unroll
  for (int r = 0; r < 3; ++r) d[r] = A.Rc[r] * dc0 + A.Rc[3 + r] * dc1 + A.Rc[6 + r] * dc2;
}

// Nearest box hit at t >= 1 along the ray of pixel (i, j) of instance `inst` (obj = -1: none);
// box frames from shared memory (sf) when staged, else computed here.
__device__ Hit trace(const CamArgs& A, const float* __restrict__ state, const BoxFrame* sf, bool staged, int inst, int i,
                     int j) {
  float d[3], x = 0.f, y = 0.f;
  if (staged) {  // the pixel's camera coordinates (per-object directions from the staged e)
    x = A.pf * (((float)j + 0.5f) - 0.5f * (float)A.W);
    y = A.pf * (((float)i + 0.5f) - 0.5f * (float)A.H);
  } else {
    ray_dir(A, i, j, d);
  }
  Hit h;
  h.obj = -1;
  h.k = 0;
  h.t = INFINITY;
  for (int o = 0; o < A.n_obj; ++o) {
    if (staged && ((float)j < sf[o].rect[0] || (float)j > sf[o].rect[1] || (float)i < sf[o].rect[2] ||
                   (float)i > sf[o].rect[3]))
      continue;  // outside the object's screen rectangle: no hit
    BoxFrame F;
    float dl[3];
    if (staged) {
      F = sf[o];
#pragma unroll
      for (int k = 0; k < 3; ++k) dl[k] = fmaf(x, F.e[k], fmaf(y, F.e[3 + k], F.e[6 + k]));
    } else {
      box_frame(A, state, inst, o, F);
#pragma unroll
      for (int k = 0; k < 3; ++k) dl[k] = F.R[k] * d[0] + F.R[3 + k] * d[1] + F.R[6 + k] * d[2];
    }
    if (A.kind[o] != DP_OBJ_BOX) {
      float tn;
      int kn;
      if (A.kind[o] == DP_OBJ_SPHERE) {
        // near root of a t^2 + 2 b t + c = 0 with the discriminant as a r^2 - |d x o|^2 (no
        // cancellation when the sphere is far)
        const float r = A.half[o][0];
        const float a = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
        const float b = dl[0] * F.o[0] + dl[1] * F.o[1] + dl[2] * F.o[2];
        const float cx = dl[1] * F.o[2] - dl[2] * F.o[1], cy = dl[2] * F.o[0] - dl[0] * F.o[2],
                    cz = dl[0] * F.o[1] - dl[1] * F.o[0];
        const float disc = a * r * r - (cx * cx + cy * cy + cz * cz);
        if (!(disc >= 0.f)) continue;
        tn = (-b - sqrtf(disc)) / a;
        kn = -1;
      } else {
        if (dl[2] == 0.f) continue;
        tn = -F.o[2] / dl[2];
        kn = -2;
      }
      if (!(tn >= 1.f) || !(tn < h.t)) continue;
      h.obj = o;
      h.k = kn;
      h.t = tn;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        h.ol[k] = F.o[k];
        h.dl[k] = dl[k];
      }
      continue;
    }
    float tn = -INFINITY, tf = INFINITY;
    int kn = 0;
    bool miss = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float hk = A.half[o][k];
      if (dl[k] == 0.f) {
        if (fabsf(F.o[k]) > hk) miss = true;
        continue;
      }
      const float inv = __frcp_rn(dl[k]);  // one correctly rounded reciprocal per slab
      float t1 = (-hk - F.o[k]) * inv, t2 = (hk - F.o[k]) * inv;
      if (t1 > t2) {
        const float s = t1;
        t1 = t2;
        t2 = s;
      }
      if (t1 > tn) {
        tn = t1;
        kn = k;
      }
      tf = fminf(tf, t2);
    }
    if (miss || !(tn <= tf) || !(tn >= 1.f) || !(tn < h.t)) continue;
    h.obj = o;
    h.k = kn;
    h.t = tn;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      h.ol[k] = F.o[k];
      h.dl[k] = dl[k];
    }
  }
  return h;
}

// Texture coordinates of a hit: the hit parameter t, the hit point p in the object's frame (for a
// box face: its two in-face coordinates qa = p_a, qc = p_c), and the bilinear sample position.
struct Sample {
  int a, c;
  float s, t, qa, qc, fx, fy;
  float p[3];
  int x0, x1, y0, y1;
};

__device__ __forceinline__ Sample sample_of(const CamArgs& A, const Hit& h) {
  Sample S;
  float u, v;
  if (h.k >= 0) {
    const int k = h.k;
    S.a = (k + 1) % 3;
    S.c = (k + 2) % 3;
    const float hk = A.half[h.obj][k];
    const float dk = pick3(h.dl, k), ok = pick3(h.ol, k);
    S.s = dk > 0.f ? -1.f : 1.f;
    S.t = (S.s * hk - ok) / dk;
    S.qa = pick3(h.ol, S.a) + S.t * pick3(h.dl, S.a);
    S.qc = pick3(h.ol, S.c) + S.t * pick3(h.dl, S.c);
    u = (S.qa / A.half[h.obj][S.a] + 1.f) * 0.5f;
    v = (S.qc / A.half[h.obj][S.c] + 1.f) * 0.5f;
  } else {
    S.a = 0;
    S.c = 1;
    S.s = 0.f;
    S.t = h.t;
#pragma unroll
    for (int k = 0; k < 3; ++k) S.p[k] = h.ol[k] + S.t * h.dl[k];
    if (h.k == -1) {  // sphere: the hit direction's spherical angles in the body frame
      const float r = A.half[h.obj][0];
      u = atan2f(S.p[1], S.p[0]) * (0.5f / 3.14159265358979f) + 0.5f;
      v = acosf(fminf(fmaxf(S.p[2] / r, -1.f), 1.f)) * (1.f / 3.14159265358979f);
    } else {  // plane: in-plane coordinates, the texture repeated
      const float uu = S.p[0] / (2.f * A.half[h.obj][0]) + 0.5f, vv = S.p[1] / (2.f * A.half[h.obj][1]) + 0.5f;
      u = uu - floorf(uu);
      v = vv - floorf(vv);
    }
    S.qa = S.qc = 0.f;
  }
  const float xs = u * (float)A.tw - 0.5f, ys = v * (float)A.th - 0.5f;
  const float x0f = floorf(xs), y0f = floorf(ys);
  S.fx = xs - x0f;
  S.fy = ys - y0f;
  auto cl = [](int q, int n) { return q < 0 ? 0 : (q >= n ? n - 1 : q); };
  S.x0 = cl((int)x0f, A.tw);
  S.x1 = cl((int)x0f + 1, A.tw);
  S.y0 = cl((int)y0f, A.th);
  S.y1 = cl((int)y0f + 1, A.th);
  return S;
}

#ifndef DPK_RENDER_BLOCKS
#define DPK_RENDER_BLOCKS 6
#endif
__global__ void __launch_bounds__(kThreads, DPK_RENDER_BLOCKS) k_render(const __grid_constant__ CamArgs A, const float* __restrict__ state,
                                                     const float* __restrict__ tex, float* __restrict__ image,
                                                     int* __restrict__ hit_out) {
  __shared__ BoxFrame sf[kMaxObj];
  int inst0, pix0;
  const bool staged = stage_frames(A, state, sf, inst0, pix0);
  const int npix = A.W * A.H;
#pragma unroll 1
  for (int r = 0; r < kPixPerThread; ++r) {
    int inst, pix;
    if (!pixel_of(A, staged, inst0, pix0, r, inst, pix)) break;
    int i, j;
    pixel_ij(A, pix, i, j);
    const Hit h = trace(A, state, sf, staged, inst, i, j);
    float col[3] = {0.f, 0.f, 0.f};
    if (h.obj >= 0) {
      const Sample S = sample_of(A, h);
      const float* T = tex + (size_t)A.tex[h.obj] * A.th * A.tw * 3;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float t00 = __ldg(T + (S.y0 * A.tw + S.x0) * 3 + ch), t01 = __ldg(T + (S.y0 * A.tw + S.x1) * 3 + ch);
        const float t10 = __ldg(T + (S.y1 * A.tw + S.x0) * 3 + ch), t11 = __ldg(T + (S.y1 * A.tw + S.x1) * 3 + ch);
        col[ch] = (1.f - S.fy) * ((1.f - S.fx) * t00 + S.fx * t01) + S.fy * ((1.f - S.fx) * t10 + S.fx * t11);
      }
    }
    const size_t idx = (size_t)inst * npix + pix;
    float* o = image + idx * 3;
    o[0] = col[0];
    o[1] = col[1];
    o[2] = col[2];
    if (hit_out) hit_out[idx] = h.obj;
  }
}

// Reverse mode: dstate[inst][body][0..11] (position, rotation entries) += the pixel's share of
// d(sum dimage * image); dtex (optional) += the texel shares. A warp whose 32 pixels belong to one
// instance sums its state shares per body with shuffles before one atomic per value.
__global__ void __launch_bounds__(kThreads) k_render_bwd(const __grid_constant__ CamArgs A, const float* __restrict__ state,
                                                         const float* __restrict__ tex, const float* __restrict__ dimage,
                                                         float* __restrict__ dstate, float* __restrict__ dtex) {
  __shared__ BoxFrame sf[kMaxObj];
  int inst0s, pix0;
  const bool staged = stage_frames(A, state, sf, inst0s, pix0);
  const int npixi = A.W * A.H;
#pragma unroll 1
  for (int rr = 0; rr < kPixPerThread; ++rr) {
  int inst = -1, pixr = 0;
  const bool live = pixel_of(A, staged, inst0s, pix0, rr, inst, pixr);
  if (!live) inst = -1;
  const size_t idx = (size_t)(live ? inst : 0) * npixi + pixr;
  float g[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) g[k] = 0.f;
  int gb = -1;  // body receiving g (-1: none)
  if (live) {
    int i, j;
    pixel_ij(A, pixr, i, j);
    const Hit h = trace(A, state, sf, staged, inst, i, j);
    if (h.obj >= 0) {
      const Sample S = sample_of(A, h);
      const float* T = tex + (size_t)A.tex[h.obj] * A.th * A.tw * 3;
      const float* dI = dimage + idx * 3;
      float dfx = 0.f, dfy = 0.f;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float gi = dI[ch];
        const size_t i00 = ((size_t)S.y0 * A.tw + S.x0) * 3 + ch, i01 = ((size_t)S.y0 * A.tw + S.x1) * 3 + ch;
        const size_t i10 = ((size_t)S.y1 * A.tw + S.x0) * 3 + ch, i11 = ((size_t)S.y1 * A.tw + S.x1) * 3 + ch;
        const float t00 = __ldg(T + i00), t01 = __ldg(T + i01), t10 = __ldg(T + i10), t11 = __ldg(T + i11);
        dfx += gi * ((1.f - S.fy) * (t01 - t00) + S.fy * (t11 - t10));
        dfy += gi * (((1.f - S.fx) * t10 + S.fx * t11) - ((1.f - S.fx) * t00 + S.fx * t01));
        if (dtex && gi != 0.f) {
          float* D = dtex + (size_t)A.tex[h.obj] * A.th * A.tw * 3;
          atomicAdd(D + i00, gi * (1.f - S.fx) * (1.f - S.fy));
          atomicAdd(D + i01, gi * S.fx * (1.f - S.fy));
          atomicAdd(D + i10, gi * (1.f - S.fx) * S.fy);
          atomicAdd(D + i11, gi * S.fx * S.fy);
        }
      }
      const int b = A.body[h.obj];
      if (b >= 0) {
        BoxFrame F;
        if (staged)
          F = sf[h.obj];
        else
          box_frame(A, state, inst, h.obj, F);
        // fx = u tw - 1/2 - floor: du = dfx tw; likewise dv = dfy th
        const float gu = dfx * (float)A.tw, gv = dfy * (float)A.th;
        float dol[3], ddl[3];
        if (h.k >= 0) {
          // u = (qa / h_a + 1)/2: dqa = du / (2 h_a); likewise qc
          const float dqa = gu * 0.5f / A.half[h.obj][S.a];
          const float dqc = gv * 0.5f / A.half[h.obj][S.c];
          const float dt = dqa * pick3(h.dl, S.a) + dqc * pick3(h.dl, S.c);
          const float dk = pick3(h.dl, h.k);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            // qa = ol_a + t dl_a, qc = ol_c + t dl_c, t = (s h_k - ol_k) / dl_k
            dol[k] = (k == S.a ? dqa : 0.f) + (k == S.c ? dqc : 0.f) + (k == h.k ? -dt / dk : 0.f);
            ddl[k] = (k == S.a ? dqa * S.t : 0.f) + (k == S.c ? dqc * S.t : 0.f) + (k == h.k ? -dt * S.t / dk : 0.f);
          }
        } else {
          // adjoint of the hit point p = o + t d, then of o and d through t
          float gp[3];
          if (h.k == -1) {
            const float r = A.half[h.obj][0];
            const float rho2 = S.p[0] * S.p[0] + S.p[1] * S.p[1];
            const float cu = gu * (0.5f / 3.14159265358979f) / fmaxf(rho2, 1e-30f);
            const float zr = fminf(fmaxf(S.p[2] / r, -1.f), 1.f);
            gp[0] = -cu * S.p[1];
            gp[1] = cu * S.p[0];
            gp[2] = -gv / (3.14159265358979f * r * sqrtf(fmaxf(1e-30f, 1.f - zr * zr)));
            // a t^2 + 2 b t + c = 0: dt/do = -p / (a t + b), dt/dd = -t p / (a t + b)
            const float a = h.dl[0] * h.dl[0] + h.dl[1] * h.dl[1] + h.dl[2] * h.dl[2];
            const float b = h.dl[0] * h.ol[0] + h.dl[1] * h.ol[1] + h.dl[2] * h.ol[2];
            const float q = (gp[0] * h.dl[0] + gp[1] * h.dl[1] + gp[2] * h.dl[2]) / (a * S.t + b);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              dol[k] = gp[k] - q * S.p[k];
              ddl[k] = S.t * (gp[k] - q * S.p[k]);
            }
          } else {
            gp[0] = gu * 0.5f / A.half[h.obj][0];
            gp[1] = gv * 0.5f / A.half[h.obj][1];
            // t = -o_z / d_z: dt/do_z = -1 / d_z, dt/dd_z = -t / d_z
            const float q = (gp[0] * h.dl[0] + gp[1] * h.dl[1]) / h.dl[2];
            dol[0] = gp[0];
            dol[1] = gp[1];
            dol[2] = -q;
            ddl[0] = S.t * gp[0];
            ddl[1] = S.t * gp[1];
            ddl[2] = -q * S.t;
          }
        }
        float d[3];
        ray_dir(A, i, j, d);
        // ol_k = sum_r R[r][k] (C_r - cw_r), dl_k = sum_r R[r][k] d_r, cw = p + R c
        float dcw[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          dcw[r] = -(F.R[3 * r] * dol[0] + F.R[3 * r + 1] * dol[1] + F.R[3 * r + 2] * dol[2]);
#pragma unroll
          for (int k = 0; k < 3; ++k) g[3 + 3 * r + k] += dol[k] * (A.C[r] - F.cw[r]) + ddl[k] * d[r];
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          g[r] += dcw[r];
#pragma unroll
          for (int m = 0; m < 3; ++m) g[3 + 3 * r + m] += dcw[r] * A.cen[h.obj][m];
        }
        gb = b;
      }
    }
  }
  const unsigned full = 0xffffffffu;
  const int inst0 = __shfl_sync(full, inst, 0);
  if (__all_sync(full, inst == inst0) && inst0 >= 0) {
    for (int b = 0; b < A.nb; ++b) {
      if (!__any_sync(full, gb == b)) continue;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        float v = gb == b ? g[k] : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(full, v, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(dstate + ((size_t)inst0 * A.nb + b) * 18 + k, v);
      }
    }
  } else if (gb >= 0) {
#pragma unroll
    for (int k = 0; k < 12; ++k) atomicAdd(dstate + ((size_t)inst * A.nb + gb) * 18 + k, g[k]);
  }
  }
}

thread_local std::string g_cam_err;

dp_status cam_args(const dp_camera* cam, const dp_scene* sc, int32_t B, int32_t nb, CamArgs& A) {
  if (!cam || !sc) { g_cam_err = "camera or scene is NULL"; return DP_EINVAL; }
  if (cam->width < 1 || cam->height < 1 || !(cam->focal > 0.f) || !(cam->plane > 0.f)) {
    g_cam_err = "camera: width, height, focal and plane must be positive";
    return DP_EINVAL;
  }
  if ((long long)cam->width * cam->height >= (1LL << 24)) {
    g_cam_err = "camera: width * height must be below 2^24 pixels";
    return DP_EINVAL;
  }
  if (B < 0 || nb < 0 || sc->n_obj < 0 || sc->n_obj > kMaxObj) {
    g_cam_err = "scene: n_obj out of range [0, DP_CAMERA_MAX_OBJECTS], or a negative size";
    return DP_EINVAL;
  }
  if (sc->n_obj > 0 && (!sc->body || !sc->center || !sc->half || !sc->tex)) {
    g_cam_err = "scene arrays are required when n_obj > 0";
    return DP_EINVAL;
  }
  if (sc->tex_h < 1 || sc->tex_w < 1 || sc->n_tex < 1) { g_cam_err = "scene: texture sizes must be >= 1"; return DP_EINVAL; }
  A.W = cam->width;
  A.H = cam->height;
  A.B = B;
  A.nb = nb;
  A.n_obj = sc->n_obj;
  A.th = sc->tex_h;
  A.tw = sc->tex_w;
  A.f = cam->focal;
  A.plane = cam->plane;
  A.pf = cam->plane / cam->focal;
  A.invW = 1.f / (float)cam->width;
  A.cull = getenv("DP_CAMERA_NO_CULL") ? 0 : 1;
  for (int k = 0; k < 3; ++k) A.C[k] = cam->position[k];
  for (int k = 0; k < 9; ++k) A.Rc[k] = cam->rotation[k];
  for (int o = 0; o < sc->n_obj; ++o) {
    if (sc->body[o] < -1 || sc->body[o] >= nb) { g_cam_err = "scene: object body out of range"; return DP_EINVAL; }
    if (sc->tex[o] < 0 || sc->tex[o] >= sc->n_tex) { g_cam_err = "scene: object texture out of range"; return DP_EINVAL; }
    A.body[o] = sc->body[o];
    A.tex[o] = sc->tex[o];
    A.kind[o] = sc->kind ? sc->kind[o] : DP_OBJ_BOX;
    if (A.kind[o] < DP_OBJ_BOX || A.kind[o] > DP_OBJ_PLANE) { g_cam_err = "scene: unknown object kind"; return DP_EINVAL; }
    for (int k = 0; k < 3; ++k) {
      A.cen[o][k] = sc->center[3 * o + k];
      A.half[o][k] = sc->half[3 * o + k];
      if (!(A.half[o][k] > 0.f)) { g_cam_err = "scene: half extents must be positive"; return DP_EINVAL; }
    }
  }
  return DP_OK;
}

}  // namespace

extern "C" {

dp_status dp_render(const dp_camera* cam, const dp_scene* scene, int32_t n_instances, int32_t n_bodies,
                    const float* state, const float* textures, float* image, int32_t* hit, void* stream) {
  CamArgs A;
  dp_status st = cam_args(cam, scene, n_instances, n_bodies, A);
  if (st != DP_OK) return st;
  if (!state || !textures || !image) { g_cam_err = "state, textures and image are required"; return DP_EINVAL; }
  const size_t n = (size_t)A.W * A.H * A.B;
  if (n == 0) return DP_OK;
  k_render<<<(unsigned)((n + kChunk - 1) / kChunk), kThreads, 0, (cudaStream_t)stream>>>(A, state, textures, image, hit);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { g_cam_err = cudaGetErrorString(e); return DP_ECUDA; }
  return DP_OK;
}

dp_status dp_render_backward(const dp_camera* cam, const dp_scene* scene, int32_t n_instances, int32_t n_bodies,
                             const float* state, const float* textures, const float* dimage, float* dstate,
                             float* dtextures, void* stream) {
  CamArgs A;
  dp_status st = cam_args(cam, scene, n_instances, n_bodies, A);
  if (st != DP_OK) return st;
  if (!state || !textures || !dimage || !dstate) { g_cam_err = "state, textures, dimage and dstate are required"; return DP_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(dstate, 0, sizeof(float) * (size_t)A.B * A.nb * 18, s);
  if (e == cudaSuccess && dtextures)
    e = cudaMemsetAsync(dtextures, 0, sizeof(float) * (size_t)scene->n_tex * A.th * A.tw * 3, s);
  const size_t n = (size_t)A.W * A.H * A.B;
  if (e == cudaSuccess && n > 0) {
    k_render_bwd<<<(unsigned)((n + kChunk - 1) / kChunk), kThreads, 0, s>>>(A, state, textures, dimage, dstate, dtextures);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { g_cam_err = cudaGetErrorString(e); return DP_ECUDA; }
  return DP_OK;
}

const char* dp_camera_last_error(void) { return g_cam_err.c_str(); }

}  // extern "C"
