// The force-controlled local relaxation of every set (Eqs. 15-18), around the
// set solve of relax.cu.
//
// Eq. 16 keeps the forces from the outer region constant: the set is cut free
// (k^Inner + Delta k of Eq. 15 is the stiffness of the set's own bars), and
// subtracting (k^Inner + Delta k) u^Inner-old from both sides gives the
// increment of Eq. 17 from the global residual: (k^Inner + Delta k) delta^RF =
// r_I.  A set clear of the supports can move rigidly, so the matrix is
// singular; reading (as the oracle's): delta^RF is the minimum-norm solution of
// the system with r_I projected onto the matrix's range.  The rigid motions
// the supports leave free span the null space N = R C (R: the translations and
// the rotation about the set's representing point, C: the combinations that
// vanish on the set's constrained DOFs), and with M = C (N^T N)^-1 C^T the
// projection onto it is R M R^T.  So:
//
//   k_force_in   r_p = r_I - R M R^T r_I, and 0 at the pinned DOFs;
//   (relax.cu)   delta_p = A_pin^-1 r_p with the cut-free factor whose pinned
//                DOFs (one per free rigid motion, chosen so that N restricted to
//                them is invertible) are unit rows: the solution of A delta =
//                r_p that vanishes there, since r_p is orthogonal to N;
//   k_force_out  delta^RF = delta_p - R M R^T delta_p (the minimum-norm one),
//                and the upper-level forces of the modes 10-12 of Eqs. 17-18,
//                P = sum delta^RF . r, sum xi delta^RF . r, sum eta delta^RF . r
//                (Eq. 7 with the FP64 residual).
//
// One CTA per set; every sum runs in a fixed order (node order per thread,
// then a fixed-shape tree), so the results are the same on every run.
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "hms_internal.cuh"

namespace hms {
namespace {

constexpr int NT = 256;

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// Deterministic sum of N values over the CTA; the totals land in tot[0..N).
template <int N>
__device__ inline void cta_sum(double (&v)[N], double* red, double* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const double w = warp_sum(v[k]);
    if (lane == 0) red[warp * N + k] = w;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double t = 0.0;
    for (int ww = 0; ww < NT / 32; ++ww) t += red[ww * N + threadIdx.x];
    tot[threadIdx.x] = t;
  }
  __syncthreads();
}

template <typename T2>
__device__ inline double2 ld2(const T2* p, size_t n);
template <>
__device__ inline double2 ld2<double2>(const double2* p, size_t n) { return p[n]; }
template <>
__device__ inline double2 ld2<float2>(const float2* p, size_t n) {
  const float2 f = p[n];
  return make_double2((double)f.x, (double)f.y);
}
template <typename T2>
__device__ inline void st2(T2* p, size_t n, double2 v);
template <>
__device__ inline void st2<double2>(double2* p, size_t n, double2 v) { p[n] = v; }
template <>
__device__ inline void st2<float2>(float2* p, size_t n, double2 v) { p[n] = make_float2((float)v.x, (float)v.y); }

__global__ void __launch_bounds__(NT) k_force_in(LatView lv, const double2* __restrict__ r,
                                                 const double* __restrict__ M, const uint8_t* __restrict__ fixF,
                                                 double2* __restrict__ rp, const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  __shared__ double red[(NT / 32) * 3], tot[3];
  const int I = blockIdx.x;
  const int i0 = (I % lv.Mx) * lv.sx, j0 = (I / lv.Mx) * lv.sy;
  const int w = min(lv.sx, lv.nx - i0), h = min(lv.sy, lv.ny - j0);
  const double2 c = lv.rep[I];
  const double* MI = M + 9 * (size_t)I;
  double s[3] = {0.0, 0.0, 0.0};
  // R^T r over the set's free DOFs (r is 0 on constrained ones)
  for (int q = threadIdx.x; q < w * h; q += NT) {
    const int i = i0 + q % w, j = j0 + q / w;
    const double2 v = r[(size_t)j * lv.nx + i];
    const double xi = node_x(lv, i, j) - c.x, eta = node_y(lv, j) - c.y;
    s[0] += v.x;
    s[1] += v.y;
    s[2] = fma(xi, v.y, fma(-eta, v.x, s[2]));
  }
  cta_sum<3>(s, red, tot);
  const double g0 = MI[0] * tot[0] + MI[1] * tot[1] + MI[2] * tot[2];
  const double g1 = MI[3] * tot[0] + MI[4] * tot[1] + MI[5] * tot[2];
  const double g2 = MI[6] * tot[0] + MI[7] * tot[1] + MI[8] * tot[2];
  for (int q = threadIdx.x; q < w * h; q += NT) {
    const int i = i0 + q % w, j = j0 + q / w;
    const size_t n = (size_t)j * lv.nx + i;
    const double2 v = r[n];
    const double xi = node_x(lv, i, j) - c.x, eta = node_y(lv, j) - c.y;
    const unsigned fm = lv.fix[n], fp = fixF[n];
    double2 o;
    o.x = (fm & 1u) ? 0.0 : v.x - fma(-g2, eta, g0);
    o.y = (fm & 2u) ? 0.0 : v.y - fma(g2, xi, g1);
    if (fp & 1u) o.x = 0.0;  // pinned (or constrained): the row is not part of the system
    if (fp & 2u) o.y = 0.0;
    rp[n] = o;
  }
}

template <typename T2>
__global__ void __launch_bounds__(NT) k_force_out(LatView lv, T2* __restrict__ d, const double* __restrict__ M,
                                                  const double2* __restrict__ r, double* __restrict__ P,
                                                  const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  __shared__ double red[(NT / 32) * 3], tot[3];
  const int I = blockIdx.x;
  const int i0 = (I % lv.Mx) * lv.sx, j0 = (I / lv.Mx) * lv.sy;
  const int w = min(lv.sx, lv.nx - i0), h = min(lv.sy, lv.ny - j0);
  const double2 c = lv.rep[I];
  const double* MI = M + 9 * (size_t)I;
  double s[3] = {0.0, 0.0, 0.0};
  for (int q = threadIdx.x; q < w * h; q += NT) {
    const int i = i0 + q % w, j = j0 + q / w;
    const double2 v = ld2(d, (size_t)j * lv.nx + i);
    const double xi = node_x(lv, i, j) - c.x, eta = node_y(lv, j) - c.y;
    s[0] += v.x;
    s[1] += v.y;
    s[2] = fma(xi, v.y, fma(-eta, v.x, s[2]));
  }
  cta_sum<3>(s, red, tot);
  const double g0 = MI[0] * tot[0] + MI[1] * tot[1] + MI[2] * tot[2];
  const double g1 = MI[3] * tot[0] + MI[4] * tot[1] + MI[5] * tot[2];
  const double g2 = MI[6] * tot[0] + MI[7] * tot[1] + MI[8] * tot[2];
  double p[3] = {0.0, 0.0, 0.0};
  for (int q = threadIdx.x; q < w * h; q += NT) {
    const int i = i0 + q % w, j = j0 + q / w;
    const size_t n = (size_t)j * lv.nx + i;
    const double2 v = ld2(d, n);
    const double xi = node_x(lv, i, j) - c.x, eta = node_y(lv, j) - c.y;
    const unsigned fm = lv.fix[n];
    double2 o;
    o.x = (fm & 1u) ? 0.0 : v.x - fma(-g2, eta, g0);
    o.y = (fm & 2u) ? 0.0 : v.y - fma(g2, xi, g1);
    st2(d, n, o);
    // P of the modes 10-12 from the delta as stored (FP32 on the mixed path)
    const double2 os = ld2(d, n);
    const double2 rv = r[n];
    const double dr = fma(os.x, rv.x, os.y * rv.y);
    p[0] += dr;
    p[1] = fma(xi, dr, p[1]);
    p[2] = fma(eta, dr, p[2]);
  }
  __syncthreads();  // tot is reused
  cta_sum<3>(p, red, tot);
  if (threadIdx.x < 3) P[(size_t)lv.q * I + 9 + threadIdx.x] = tot[threadIdx.x];
}

}  // namespace

cudaError_t launch_force_in(cudaStream_t s, const LatView& lv, const double2* r, const double* M,
                            const uint8_t* fixF, double2* rproj, const IterCtl* ctl) {
  k_force_in<<<lv.M, NT, 0, s>>>(lv, r, M, fixF, rproj, ctl);
  return cudaGetLastError();
}

cudaError_t launch_force_out(cudaStream_t s, const LatView& lv, void* drf, bool fp32, const double* M,
                             const double2* r, double* P, const IterCtl* ctl) {
  if (fp32) k_force_out<float2><<<lv.M, NT, 0, s>>>(lv, (float2*)drf, M, r, P, ctl);
  else k_force_out<double2><<<lv.M, NT, 0, s>>>(lv, (double2*)drf, M, r, P, ctl);
  return cudaGetLastError();
}

}  // namespace hms

// ---------------------------------------------------------------- host: per-set data
namespace hms {
namespace {
// eigenvalues / eigenvectors (columns of V) of a symmetric 3 x 3 matrix, Jacobi rotations
void eig3(double A[3][3], double w[3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    if (off < 1e-300) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        const double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; ++k) {  // A <- A G on columns p, q
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- G^T A on rows p, q
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < 3; ++i) w[i] = A[i][i];
}
double det_small(const double* a, int d) {  // d x d row-major, d <= 3
  if (d == 1) return a[0];
  if (d == 2) return a[0] * a[3] - a[1] * a[2];
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
}
void inv_small(const double* a, double* out, int d) {
  const double det = det_small(a, d);
  if (d == 1) {
    out[0] = 1.0 / a[0];
  } else if (d == 2) {
    out[0] = a[3] / det, out[1] = -a[1] / det, out[2] = -a[2] / det, out[3] = a[0] / det;
  } else {
    out[0] = (a[4] * a[8] - a[5] * a[7]) / det;
    out[1] = (a[2] * a[7] - a[1] * a[8]) / det;
    out[2] = (a[1] * a[5] - a[2] * a[4]) / det;
    out[3] = (a[5] * a[6] - a[3] * a[8]) / det;
    out[4] = (a[0] * a[8] - a[2] * a[6]) / det;
    out[5] = (a[2] * a[3] - a[0] * a[5]) / det;
    out[6] = (a[3] * a[7] - a[4] * a[6]) / det;
    out[7] = (a[1] * a[6] - a[0] * a[7]) / det;
    out[8] = (a[0] * a[4] - a[1] * a[3]) / det;
  }
}
}  // namespace

// Per set: the projection matrix M (row-major 3 x 3) onto the rigid motions
// R C the set's supports leave free (R: rows (1, 0, -eta) for an x DOF and
// (0, 1, xi) for a y DOF; C: a basis of the combinations vanishing on the
// constrained DOFs), and the pinned DOFs added to fixF: as many as there are
// free rigid motions, among the free DOFs of the set's corner nodes, the
// choice whose rows of R C have the largest |determinant|.  False if a set's
// free rigid motions cannot be pinned there.
bool force_set_data(const LatView& lv, const std::vector<uint8_t>& fix, const std::vector<double2>& rep,
                    std::vector<double>& M, std::vector<uint8_t>& fixF) {
  M.assign(9 * (size_t)lv.M, 0.0);
  fixF = fix;
  for (int I = 0; I < lv.M; ++I) {
    const int i0 = (I % lv.Mx) * lv.sx, j0 = (I / lv.Mx) * lv.sy;
    const int w = std::min(lv.sx, lv.nx - i0), h = std::min(lv.sy, lv.ny - j0);
    const double cx = rep[I].x, cy = rep[I].y;
    double G[3][3] = {}, H[3][3] = {};
    auto row_of = [&](int i, int j, int c, double* r) {
      const double xi = lv.L * ((double)i + 0.5 * (double)(j & 1)) - cx, eta = lv.L * SQ3_2 * (double)j - cy;
      r[0] = c == 0 ? 1.0 : 0.0;
      r[1] = c == 1 ? 1.0 : 0.0;
      r[2] = c == 0 ? -eta : xi;
    };
    for (int j = j0; j < j0 + h; ++j)
      for (int i = i0; i < i0 + w; ++i)
        for (int c = 0; c < 2; ++c) {
          double r[3];
          row_of(i, j, c, r);
          const bool con = (fix[(size_t)j * lv.nx + i] >> c) & 1u;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) (con ? G : H)[a][b] += r[a] * r[b];
        }
    double w3[3], V[3][3];
    eig3(G, w3, V);
    const double scale = std::max(H[0][0] + H[1][1] + H[2][2], 1.0);
    double Cb[3][3];
    int d = 0;
    for (int k = 0; k < 3; ++k)
      if (std::fabs(w3[k]) <= 1e-12 * scale) {
        for (int a = 0; a < 3; ++a) Cb[a][d] = V[a][k];
        ++d;
      }
    if (d == 0) continue;  // anchored: no projection, no pin
    // N^T N = Cb^T H Cb, M = Cb (N^T N)^-1 Cb^T
    double NtN[9], NtNi[9];
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double v = 0.0;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) v += Cb[p][a] * H[p][q] * Cb[q][b];
        NtN[a * d + b] = v;
      }
    inv_small(NtN, NtNi, d);
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) {
        double v = 0.0;
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) v += Cb[p][a] * NtNi[a * d + b] * Cb[q][b];
        M[9 * (size_t)I + 3 * p + q] = v;
      }
    // pins: free DOFs of the corner nodes
    std::vector<std::array<int, 3>> cand;  // i, j, c
    const int ci[4] = {i0, i0 + w - 1, i0, i0 + w - 1}, cj[4] = {j0, j0, j0 + h - 1, j0 + h - 1};
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 2; ++c)
        if (!((fix[(size_t)cj[k] * lv.nx + ci[k]] >> c) & 1u)) cand.push_back({ci[k], cj[k], c});
    double best = 0.0;
    int pick[3] = {-1, -1, -1};
    const int nc = (int)cand.size();
    for (int a = 0; a < nc; ++a)
      for (int b = (d > 1 ? a + 1 : a); b < (d > 1 ? nc : a + 1); ++b)
        for (int e = (d > 2 ? b + 1 : b); e < (d > 2 ? nc : b + 1); ++e) {
          const int sel[3] = {a, b, e};
          double m[9];
          for (int r = 0; r < d; ++r) {
            double rr[3];
            row_of(cand[sel[r]][0], cand[sel[r]][1], cand[sel[r]][2], rr);
            for (int cc = 0; cc < d; ++cc) m[r * d + cc] = rr[0] * Cb[0][cc] + rr[1] * Cb[1][cc] + rr[2] * Cb[2][cc];
          }
          const double dt = std::fabs(det_small(m, d));
          if (dt > best) best = dt, pick[0] = a, pick[1] = b, pick[2] = e;
        }
    if (!(best > 1e-9)) return false;
    for (int r = 0; r < d; ++r) {
      const auto& cd = cand[pick[r]];
      fixF[(size_t)cd[1] * lv.nx + cd[0]] |= (uint8_t)(1u << cd[2]);
    }
  }
  return true;
}

}  // namespace hms
