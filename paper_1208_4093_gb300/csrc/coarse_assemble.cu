// K3: the upper-level matrix K_aa = V^T K V of Eq. 6, and its band storage.
//
// K = sum over bars of (EA/L) g g^T with g = e at the owner's DOFs and -e at
// the other end's, so a bar adds (EA/L) s s^T to K_aa, where s_m = e . (V_m(a)
// - V_m(b)) over the modes of the (at most two) sets the bar touches.  A bar
// inside set I touches only I's nine modes; a bar crossing to a neighbour set
// J touches 18 (I's at the owner a, J's at b with a minus sign).
//
// One CTA per set I sums the bars owned by its nodes into six 18 x 18 slots:
// SELF (bars inside I, upper-left 9 x 9 used) and E, W, N, NE, NW (bars to the
// neighbour set in that direction; rows/cols 0-8 = I's modes, 9-17 = J's).
// The translation/gradient entries (modes 1-6) do not depend on delta: they
// are summed once at setup (FULL = true, delta = 0) into a base copy, and
// every iteration only the entries that involve modes 7-9 are summed
// (FULL = false).  For bars inside I with all four DOFs free the translation
// terms vanish and the gradient terms are constants of the bar direction, so
// those bars only accumulate e.delta sums per direction; bars touching a
// constrained DOF use the general 9-term form.  All sums run in a fixed order
// (per-thread node order, then a fixed-shape tree), so the result is the same
// on every run.
#include "hms_internal.cuh"

namespace hms {
namespace {

constexpr int NT = 256, NW = NT / 32;
constexpr int NREG = 15;          // 3 directions x 3 delta modes + 6 delta-delta products
constexpr int NGEN_DELTA = 24;    // (m, l), m in 6..8, l <= m
constexpr int NGEN_FULL = 45;     // (m, l), l <= m < 9
constexpr int LSTRIDE = 36;       // s[18], (EA/L) s[18]
constexpr int RED_CHUNK = NW;     // accumulators per shared-memory reduction pass

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

template <typename DT>
__device__ inline double2 ld_delta(const DT* d, size_t n);
template <>
__device__ inline double2 ld_delta<double2>(const double2* d, size_t n) { return d[n]; }
template <>
__device__ inline double2 ld_delta<float2>(const float2* d, size_t n) {
  const float2 f = d[n];
  return make_double2((double)f.x, (double)f.y);
}

__device__ inline int gen_idx(int m, int l, bool full) {
  if (full) return m * (m + 1) / 2 + l;
  return (m == 6 ? 0 : (m == 7 ? 7 : 15)) + l;
}

// e . V_m at a node, modes m = 0..8 (Eqs. 9, 10, 13, 14), zero on constrained DOFs.
__device__ inline void mode_proj(double ex, double ey, double xi, double eta, unsigned fm, double2 dl,
                                 double* s) {
  const double fx = (fm & 1u) ? 0.0 : 1.0, fy = (fm & 2u) ? 0.0 : 1.0;
  const double ed = ex * dl.x + ey * dl.y;  // delta is 0 on constrained DOFs
  s[0] = ex * fx;
  s[1] = ey * fy;
  s[2] = ex * xi * fx;
  s[3] = ex * eta * fx;
  s[4] = ey * xi * fy;
  s[5] = ey * eta * fy;
  s[6] = ed;
  s[7] = xi * ed;
  s[8] = eta * ed;
}

// mode_proj in the arithmetic AT of the per-bar products (the same formula)
template <typename AT>
__device__ inline void mode_proj_t(AT ex, AT ey, AT xi, AT eta, unsigned fm, AT dx, AT dy, AT* s) {
  const AT fx = (fm & 1u) ? AT(0) : AT(1), fy = (fm & 2u) ? AT(0) : AT(1);
  const AT ed = ex * dx + ey * dy;
  s[0] = ex * fx;
  s[1] = ey * fy;
  s[2] = ex * xi * fx;
  s[3] = ex * eta * fx;
  s[4] = ey * xi * fy;
  s[5] = ey * eta * fy;
  s[6] = ed;
  s[7] = xi * ed;
  s[8] = eta * ed;
}
template <typename AT>
__device__ inline AT warp_sum_t(AT v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

struct ListCaps {
  int cap[6], off[6], total;
};
__host__ __device__ inline ListCaps list_caps(int w, int h) {
  ListCaps c;
  c.cap[SLOT_SELF] = 0;
  c.cap[SLOT_E] = 2 * h;
  c.cap[SLOT_W] = h;
  c.cap[SLOT_N] = 2 * w;
  c.cap[SLOT_NE] = 2;
  c.cap[SLOT_NW] = 2;
  int o = 0;
  for (int k = 0; k < 6; ++k) {
    c.off[k] = o;
    o += c.cap[k];
  }
  c.total = o;
  return c;
}

// AT: arithmetic of the per-bar products (double on the FP64 path; float on
// the mixed path, where delta itself is FP32 and the products only
// approximate K_aa, which leaves the iteration's fixed point unchanged because
// P uses the FP64 residual).  On the mixed path the interface bars' products,
// the sums over a slot's bars (in chunks of 16, the chunks added in FP64) and
// the block reduction of the per-thread sums run in FP32 too; on the FP64
// path everything is FP64.
// The kernel body for set I.
template <typename DT, bool FULL, typename AT>
__device__ __forceinline__ void slots_body(const LatView lv, const DT* __restrict__ delta, double* __restrict__ slots,
                                           const IterCtl* ctl, int I) {
  extern __shared__ double lists[];
  if (ctl && *(volatile const int*)&ctl->done) return;
  constexpr int NGEN = FULL ? NGEN_FULL : NGEN_DELTA;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Ix = I % lv.Mx, Iy = I / lv.Mx;
  const int i0 = Ix * lv.sx, j0 = Iy * lv.sy;
  const int w = min(lv.sx, lv.nx - i0), h = min(lv.sy, lv.ny - j0);
  const ListCaps LC = list_caps(w, h);
  double* out = slots + (size_t)I * NSLOTS * SLOT_SIZE;

  AT* la = reinterpret_cast<AT*>(lists);  // the interface lists, in AT
  for (int q = tid; q < LC.total * LSTRIDE; q += NT) la[q] = AT(0);
  for (int q = tid; q < NSLOTS * SLOT_SIZE; q += NT) out[q] = 0.0;
  __syncthreads();

  const double2 repI = lv.rep[I];
  // set-relative coordinates of the regular-bar path in AT: xi = L (il + off/2) + c0x,
  // eta = L sqrt3/2 jl + c0y; the far end of a bar of direction d adds (L e_x, L e_y)
  const AT c0x = (AT)fma(lv.L, (double)i0, -repI.x), c0y = (AT)fma(lv.L * SQ3_2, (double)j0, -repI.y);
  const AT LA = (AT)lv.L, LyA = (AT)(lv.L * SQ3_2);
  AT reg[NREG];
  AT gen[NGEN];
#pragma unroll
  for (int k = 0; k < NREG; ++k) reg[k] = AT(0);
#pragma unroll
  for (int k = 0; k < NGEN; ++k) gen[k] = AT(0);

  for (int q = tid; q < w * h; q += NT) {
    const int il = q % w, jl = q / w;
    const int i = i0 + il, j = j0 + jl;
    const int off = j & 1;
    const size_t na = (size_t)j * lv.nx + i;
    const unsigned fa = lv.fix[na];
    const DT dra = FULL ? DT{} : delta[na];
    const AT xiaA = fma(LA, (AT)il + (off ? AT(0.5) : AT(0)), c0x), etaaA = fma(LyA, (AT)jl, c0y);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double k = bar_k(lv, i, j, d);
      if (__double_as_longlong(k) == 0) continue;  // no bar (bar_k returns +0.0; EA > 0): an integer test
      const int ib = (d == 0) ? i + 1 : (d == 1 ? i + off : i - 1 + off);
      const int jb = (d == 0) ? j : j + 1;
      const size_t nbn = (size_t)jb * lv.nx + ib;
      const unsigned fb = lv.fix[nbn];
      const double ex = (d == 0) ? 1.0 : (d == 1 ? 0.5 : -0.5), ey = (d == 0) ? 0.0 : SQ3_2;
      const int dxs = (ib >= i0 + w) ? 1 : (ib < i0 ? -1 : 0);
      const int dys = (jb >= j0 + h) ? 1 : 0;
      // FP64 node data of the general and interface paths (not of regular bars)
      auto fp64_ends = [&](double2& da, double2& db, double& xa, double& ya, double& xb, double& yb) {
        da = FULL ? make_double2(0.0, 0.0) : ld_delta(delta, na);
        db = FULL ? make_double2(0.0, 0.0) : ld_delta(delta, nbn);
        xa = node_x(lv, i, j), ya = node_y(lv, j);
        xb = node_x(lv, ib, jb), yb = node_y(lv, jb);
      };
      if (dxs == 0 && dys == 0) {
        if (!FULL && fa == 0u && fb == 0u) {
          // regular bar: s_0 = s_1 = 0, s_2..s_5 constants of the direction;
          // everything in AT from the raw delta
          const DT drb = delta[nbn];
          const AT exA = (AT)ex, eyA = (AT)ey;
          const AT ea = fma(eyA, (AT)dra.y, exA * (AT)dra.x), eb = fma(eyA, (AT)drb.y, exA * (AT)drb.x);
          const AT xibA = fma(LA, exA, xiaA), etabA = (d == 0) ? etaaA : etaaA + LyA;
          const AT s6 = ea - eb;
          const AT s7 = fma(xiaA, ea, -(xibA * eb));
          const AT s8 = fma(etaaA, ea, -(etabA * eb));
          const AT kk = (AT)k;
          const AT k6 = kk * s6, k7 = kk * s7, k8 = kk * s8;
          reg[3 * d + 0] += k6;
          reg[3 * d + 1] += k7;
          reg[3 * d + 2] += k8;
          reg[9] = fma(k6, s6, reg[9]);
          reg[10] = fma(k7, s6, reg[10]);
          reg[11] = fma(k8, s6, reg[11]);
          reg[12] = fma(k7, s7, reg[12]);
          reg[13] = fma(k8, s7, reg[13]);
          reg[14] = fma(k8, s8, reg[14]);
        } else {
          double2 da, db;
          double xa, ya, xb, yb;
          fp64_ends(da, db, xa, ya, xb, yb);
          const double xia = xa - repI.x, etaa = ya - repI.y;
          const double xib = xb - repI.x, etab = yb - repI.y;
          double sa[9], sb[9];
          mode_proj(ex, ey, xia, etaa, fa, da, sa);
          mode_proj(ex, ey, xib, etab, fb, db, sb);
#pragma unroll
          for (int m = 0; m < 9; ++m) sa[m] -= sb[m];
          if (FULL) {
#pragma unroll
            for (int m = 0; m < 9; ++m)
#pragma unroll
              for (int l = 0; l <= m; ++l)
                gen[m * (m + 1) / 2 + l] = fma((AT)(k * sa[m]), (AT)sa[l], gen[m * (m + 1) / 2 + l]);
          } else {
#pragma unroll
            for (int m = 6; m < 9; ++m)
#pragma unroll
              for (int l = 0; l <= m; ++l) {
                const int g = (m == 6 ? 0 : (m == 7 ? 7 : 15)) + l;
                gen[g] = fma((AT)(k * sa[m]), (AT)sa[l], gen[g]);
              }
          }
        }
      }
      // else an interface bar: the pass below
    }
  }

  // Interface bars (the far end in a neighbour set), apart from the node loop
  // so that whole warps take their FP64 work (in the node loop one lane of a
  // warp would, while the FP64 pipe spends a warp instruction's full time):
  // the right column's E and NE bars, the left column's NW bars, the top
  // row's NE and NW bars.  Each list entry is written by one item; the sums
  // over the lists below are unchanged.
  for (int t = tid; t < 3 * h + 2 * w; t += NT) {
    int il, jl, d;
    if (t < 2 * h) {
      il = w - 1, jl = t >> 1, d = t & 1;
    } else if (t < 3 * h) {
      il = 0, jl = t - 2 * h, d = 2;
    } else {
      const int u = t - 3 * h;
      il = u >> 1, jl = h - 1, d = 1 + (u & 1);
      if ((d == 1 && il == w - 1) || (d == 2 && il == 0)) continue;  // in the column groups
    }
    const int i = i0 + il, j = j0 + jl, off = j & 1;
    const double k = bar_k(lv, i, j, d);
    if (__double_as_longlong(k) == 0) continue;
    const int ib = (d == 0) ? i + 1 : (d == 1 ? i + off : i - 1 + off);
    const int jb = (d == 0) ? j : j + 1;
    const int dxs = (ib >= i0 + w) ? 1 : (ib < i0 ? -1 : 0);
    const int dys = (jb >= j0 + h) ? 1 : 0;
    if (dxs == 0 && dys == 0) continue;  // an inner bar (node loop)
    const size_t na = (size_t)j * lv.nx + i, nbn = (size_t)jb * lv.nx + ib;
    const unsigned fa = lv.fix[na], fb = lv.fix[nbn];
    const double ex = (d == 0) ? 1.0 : (d == 1 ? 0.5 : -0.5), ey = (d == 0) ? 0.0 : SQ3_2;
    auto fp64_ends = [&](double2& da, double2& db, double& xa, double& ya, double& xb, double& yb) {
      da = FULL ? make_double2(0.0, 0.0) : ld_delta(delta, na);
      db = FULL ? make_double2(0.0, 0.0) : ld_delta(delta, nbn);
      xa = node_x(lv, i, j), ya = node_y(lv, j);
      xb = node_x(lv, ib, jb), yb = node_y(lv, jb);
    };
    {
      int slot, idx;
      if (dys == 0) {
        if (dxs > 0) {
          slot = SLOT_E;
          idx = 2 * jl + (d == 1 ? 1 : 0);
        } else {
          slot = SLOT_W;
          idx = jl;
        }
      } else if (dxs == 0) {
        slot = SLOT_N;
        idx = 2 * il + (d == 2 ? 1 : 0);
      } else if (dxs > 0) {
        slot = SLOT_NE;
        idx = (d == 1) ? 0 : 1;
      } else {
        slot = SLOT_NW;
        idx = (d == 2) ? 0 : 1;
      }
      double2 da, db;
      double xa, ya, xb, yb;
      fp64_ends(da, db, xa, ya, xb, yb);
      const int Jx = Ix + dxs, Jy = Iy + dys;
      const double2 repJ = lv.rep[Jy * lv.Mx + Jx];
      AT* e = la + (size_t)(LC.off[slot] + idx) * LSTRIDE;
      AT sa[9], sb[9];
      mode_proj_t<AT>((AT)ex, (AT)ey, (AT)(xa - repI.x), (AT)(ya - repI.y), fa, (AT)da.x, (AT)da.y, sa);
      mode_proj_t<AT>((AT)ex, (AT)ey, (AT)(xb - repJ.x), (AT)(yb - repJ.y), fb, (AT)db.x, (AT)db.y, sb);
      const AT kA = (AT)k;
#pragma unroll
      for (int m = 0; m < 9; ++m) {
        e[m] = sa[m];
        e[9 + m] = -sb[m];
        e[18 + m] = kA * sa[m];
        e[27 + m] = -(kA * sb[m]);
      }
    }
  }

  // deterministic block sums of the per-thread accumulators, eight at a time
  // through shared memory: warp a adds accumulator a of the CTA's threads
  // lane by lane in thread order, then a shuffle tree finishes it
  constexpr int NACC = NREG + NGEN;
  double* red = lists + (size_t)LC.total * LSTRIDE;  // RED_CHUNK x NT
  double* tot = red + RED_CHUNK * NT;                 // NACC CTA totals
  AT* redA = reinterpret_cast<AT*>(red);
#pragma unroll
  for (int c0 = 0; c0 < NACC; c0 += RED_CHUNK) {
#pragma unroll
    for (int q = 0; q < RED_CHUNK; ++q) {
      const int k = c0 + q;
      if (k < NREG) redA[q * NT + tid] = reg[k];
      else if (k < NACC) redA[q * NT + tid] = gen[k - NREG];
    }
    __syncthreads();
    if (c0 + warp < NACC) {
      const AT* q = redA + warp * NT + lane;
      AT v = q[0];
#pragma unroll
      for (int ww = 1; ww < NW; ++ww) v += q[32 * ww];
      v = warp_sum_t<AT>(v);
      if (lane == 0) tot[c0 + warp] = (double)v;
    }
    __syncthreads();
  }

  // SELF slot (upper-left 9 x 9)
  if (tid < 81) {
    const int m = tid / 9, l = tid % 9;
    const int mm = m > l ? m : l, ll = m > l ? l : m;
    double v = 0.0;
    bool have = false;
    if (FULL) {
      v = tot[NREG + mm * (mm + 1) / 2 + ll];
      have = true;
    } else if (mm >= 6) {
      v = tot[NREG + gen_idx(mm, ll, false)];
      const double L = lv.L;
      // constants s_2..s_5 of a regular bar of direction d: -L e_x^2, -L e_x e_y, -L e_y e_x, -L e_y^2
      if (ll >= 2 && ll <= 5) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const double ex = (d == 0) ? 1.0 : (d == 1 ? 0.5 : -0.5), ey = (d == 0) ? 0.0 : SQ3_2;
          const double c = (ll == 2) ? -L * ex * ex : (ll == 5 ? -L * ey * ey : -L * ex * ey);
          v = fma(c, tot[3 * d + (mm - 6)], v);
        }
      } else if (ll >= 6) {
        const int qi = (mm == 6) ? 9 : (mm == 7 ? (ll == 6 ? 10 : 12) : (ll == 6 ? 11 : (ll == 7 ? 13 : 14)));
        v += tot[qi];
      }
      have = true;
    }
    if (have) out[SLOT_SELF * SLOT_SIZE + m * SLOT_DIM + l] = v;
  }
  // interface slots: sum over each list in index order; each slot is
  // symmetric (a sum of (EA/L) s s^T), so only p <= c is summed
  constexpr int NUP = SLOT_DIM * (SLOT_DIM + 1) / 2;
  for (int q = tid; q < 5 * NUP; q += NT) {
    const int slot = 1 + q / NUP;
    int r = q % NUP, p = 0;
    while (r >= SLOT_DIM - p) r -= SLOT_DIM - p, ++p;
    const int c = p + r;
    const bool dp = (p % 9) >= 6, dc = (c % 9) >= 6;
    if (!FULL && !dp && !dc) continue;
    const AT* e = la + (size_t)LC.off[slot] * LSTRIDE;
    double v = 0.0;
    if constexpr (sizeof(AT) == 8) {
      for (int b = 0; b < LC.cap[slot]; ++b, e += LSTRIDE) v = fma(e[18 + p], e[c], v);
    } else {
      for (int b0 = 0; b0 < LC.cap[slot]; b0 += 16) {
        AT part = AT(0);
        for (int b = b0; b < b0 + 16 && b < LC.cap[slot]; ++b, e += LSTRIDE) part = fma(e[18 + p], e[c], part);
        v += (double)part;
      }
    }
    out[slot * SLOT_SIZE + p * SLOT_DIM + c] = v;
    out[slot * SLOT_SIZE + c * SLOT_DIM + p] = v;
  }
}

template <typename DT, bool FULL, typename AT>
__global__ void __launch_bounds__(NT) k_coarse_slots(LatView lv, const DT* __restrict__ delta,
                                                     double* __restrict__ slots, const IterCtl* ctl) {
  slots_body<DT, FULL, AT>(lv, delta, slots, ctl, blockIdx.x);
}

// ---- q = 12: the force-controlled modes 10-12 of Eqs. 17-18 as well ----
// The same bar-by-bar sums with every bar on the general path: the mode
// projections s_0..s_8 of mode_proj and s_9 = e.delta^RF, s_10 = xi s_9,
// s_11 = eta s_9; slots of 24 x 24 (rows/cols 0-11 = I's modes, 12-23 = J's).
constexpr int Q12 = NMODES_RF, SD12 = 2 * Q12, SS12 = SD12 * SD12;
constexpr int LSTRIDE12 = 4 * Q12;      // s_a, -s_b, k s_a, -k s_b
constexpr int NGEN12_FULL = 21;         // (m, l), l <= m < 6
constexpr int NGEN12_DELTA = 57;        // (m, l), m in 6..11, l <= m

__device__ inline void mode_proj12(double ex, double ey, double xi, double eta, unsigned fm, double2 dl,
                                   double2 df, double* s) {
  mode_proj(ex, ey, xi, eta, fm, dl, s);
  const double ef = ex * df.x + ey * df.y;  // delta^RF is 0 on constrained DOFs
  s[9] = ef;
  s[10] = xi * ef;
  s[11] = eta * ef;
}
__device__ inline int gen12_idx(int m, int l, bool full) {
  return full ? m * (m + 1) / 2 + l : m * (m + 1) / 2 - 21 + l;
}

template <typename DT, bool FULL, typename AT>
__device__ __forceinline__ void slots12_body(const LatView lv, const DT* __restrict__ delta,
                                             const DT* __restrict__ delta_rf, double* __restrict__ slots,
                                             const IterCtl* ctl, int I) {
  extern __shared__ double lists[];
  if (ctl && *(volatile const int*)&ctl->done) return;
  constexpr int NGEN = FULL ? NGEN12_FULL : NGEN12_DELTA;
  constexpr int MLO = FULL ? 0 : 6, MHI = FULL ? 6 : Q12;  // rows m of the sums
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Ix = I % lv.Mx, Iy = I / lv.Mx;
  const int i0 = Ix * lv.sx, j0 = Iy * lv.sy;
  const int w = min(lv.sx, lv.nx - i0), h = min(lv.sy, lv.ny - j0);
  const ListCaps LC = list_caps(w, h);
  double* out = slots + (size_t)I * NSLOTS * SS12;

  for (int q = tid; q < LC.total * LSTRIDE12; q += NT) lists[q] = 0.0;
  for (int q = tid; q < NSLOTS * SS12; q += NT) out[q] = 0.0;
  __syncthreads();

  const double2 repI = lv.rep[I];
  AT gen[NGEN];
#pragma unroll
  for (int k = 0; k < NGEN; ++k) gen[k] = AT(0);
  auto ld = [&](const DT* p, size_t n) { return FULL ? make_double2(0.0, 0.0) : ld_delta(p, n); };

  for (int q = tid; q < w * h; q += NT) {
    const int il = q % w, jl = q / w;
    const int i = i0 + il, j = j0 + jl;
    const int off = j & 1;
    const size_t na = (size_t)j * lv.nx + i;
    const unsigned fa = lv.fix[na];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double k = bar_k(lv, i, j, d);
      if (__double_as_longlong(k) == 0) continue;
      const int ib = (d == 0) ? i + 1 : (d == 1 ? i + off : i - 1 + off);
      const int jb = (d == 0) ? j : j + 1;
      if (ib >= i0 + w || ib < i0 || jb >= j0 + h) continue;  // interface bar: the pass below
      const size_t nbn = (size_t)jb * lv.nx + ib;
      const unsigned fb = lv.fix[nbn];
      const double ex = (d == 0) ? 1.0 : (d == 1 ? 0.5 : -0.5), ey = (d == 0) ? 0.0 : SQ3_2;
      double sa[Q12], sb[Q12];
      mode_proj12(ex, ey, node_x(lv, i, j) - repI.x, node_y(lv, j) - repI.y, fa, ld(delta, na), ld(delta_rf, na),
                  sa);
      mode_proj12(ex, ey, node_x(lv, ib, jb) - repI.x, node_y(lv, jb) - repI.y, fb, ld(delta, nbn),
                  ld(delta_rf, nbn), sb);
#pragma unroll
      for (int m = 0; m < Q12; ++m) sa[m] -= sb[m];
#pragma unroll
      for (int m = MLO; m < MHI; ++m)
#pragma unroll
        for (int l = 0; l <= m; ++l) {
          const int g = gen12_idx(m, l, FULL);
          gen[g] = fma((AT)(k * sa[m]), (AT)sa[l], gen[g]);
        }
    }
  }

  // interface bars (the far end in a neighbour set), as in slots_body
  for (int t = tid; t < 3 * h + 2 * w; t += NT) {
    int il, jl, d;
    if (t < 2 * h) {
      il = w - 1, jl = t >> 1, d = t & 1;
    } else if (t < 3 * h) {
      il = 0, jl = t - 2 * h, d = 2;
    } else {
      const int u = t - 3 * h;
      il = u >> 1, jl = h - 1, d = 1 + (u & 1);
      if ((d == 1 && il == w - 1) || (d == 2 && il == 0)) continue;
    }
    const int i = i0 + il, j = j0 + jl, off = j & 1;
    const double k = bar_k(lv, i, j, d);
    if (__double_as_longlong(k) == 0) continue;
    const int ib = (d == 0) ? i + 1 : (d == 1 ? i + off : i - 1 + off);
    const int jb = (d == 0) ? j : j + 1;
    const int dxs = (ib >= i0 + w) ? 1 : (ib < i0 ? -1 : 0);
    const int dys = (jb >= j0 + h) ? 1 : 0;
    if (dxs == 0 && dys == 0) continue;
    const size_t na = (size_t)j * lv.nx + i, nbn = (size_t)jb * lv.nx + ib;
    const unsigned fa = lv.fix[na], fb = lv.fix[nbn];
    const double ex = (d == 0) ? 1.0 : (d == 1 ? 0.5 : -0.5), ey = (d == 0) ? 0.0 : SQ3_2;
    int slot, idx;
    if (dys == 0) {
      if (dxs > 0) {
        slot = SLOT_E;
        idx = 2 * jl + (d == 1 ? 1 : 0);
      } else {
        slot = SLOT_W;
        idx = jl;
      }
    } else if (dxs == 0) {
      slot = SLOT_N;
      idx = 2 * il + (d == 2 ? 1 : 0);
    } else if (dxs > 0) {
      slot = SLOT_NE;
      idx = (d == 1) ? 0 : 1;
    } else {
      slot = SLOT_NW;
      idx = (d == 2) ? 0 : 1;
    }
    const int Jx = Ix + dxs, Jy = Iy + dys;
    const double2 repJ = lv.rep[Jy * lv.Mx + Jx];
    double* e = lists + (size_t)(LC.off[slot] + idx) * LSTRIDE12;
    double sa[Q12], sb[Q12];
    mode_proj12(ex, ey, node_x(lv, i, j) - repI.x, node_y(lv, j) - repI.y, fa, ld(delta, na), ld(delta_rf, na), sa);
    mode_proj12(ex, ey, node_x(lv, ib, jb) - repJ.x, node_y(lv, jb) - repJ.y, fb, ld(delta, nbn), ld(delta_rf, nbn),
                sb);
#pragma unroll
    for (int m = 0; m < Q12; ++m) {
      e[m] = sa[m];
      e[Q12 + m] = -sb[m];
      e[2 * Q12 + m] = k * sa[m];
      e[3 * Q12 + m] = -(k * sb[m]);
    }
  }

  // deterministic block sums of the per-thread accumulators, RED_CHUNK at a time
  double* red = lists + (size_t)LC.total * LSTRIDE12;  // RED_CHUNK x NT
  double* tot = red + RED_CHUNK * NT;                   // NGEN CTA totals
#pragma unroll
  for (int c0 = 0; c0 < NGEN; c0 += RED_CHUNK) {
#pragma unroll
    for (int q = 0; q < RED_CHUNK; ++q)
      if (c0 + q < NGEN) red[q * NT + tid] = (double)gen[c0 + q];
    __syncthreads();
    if (c0 + warp < NGEN) {
      const double* q = red + warp * NT + lane;
      double v = q[0];
#pragma unroll
      for (int ww = 1; ww < NW; ++ww) v += q[32 * ww];
      v = warp_sum(v);
      if (lane == 0) tot[c0 + warp] = v;
    }
    __syncthreads();
  }
  // SELF slot (upper-left 12 x 12): the entries this pass sums
  if (tid < Q12 * Q12) {
    const int m = tid / Q12, l = tid % Q12;
    const int mm = m > l ? m : l, ll = m > l ? l : m;
    if (mm >= MLO && mm < MHI) out[SLOT_SELF * SS12 + m * SD12 + l] = tot[gen12_idx(mm, ll, FULL)];
  }
  // interface slots: sums over each list in index order (symmetric: p <= c)
  constexpr int NUP = SD12 * (SD12 + 1) / 2;
  for (int q = tid; q < 5 * NUP; q += NT) {
    const int slot = 1 + q / NUP;
    int r = q % NUP, p = 0;
    while (r >= SD12 - p) r -= SD12 - p, ++p;
    const int c = p + r;
    const bool dp = (p % Q12) >= 6, dc = (c % Q12) >= 6;
    if (FULL ? (dp || dc) : (!dp && !dc)) continue;
    const double* e = lists + (size_t)LC.off[slot] * LSTRIDE12;
    double v = 0.0;
    for (int b = 0; b < LC.cap[slot]; ++b, e += LSTRIDE12) v = fma(e[2 * Q12 + p], e[c], v);
    out[slot * SS12 + p * SD12 + c] = v;
    out[slot * SS12 + c * SD12 + p] = v;
  }
}

template <typename DT, bool FULL, typename AT>
__global__ void __launch_bounds__(NT) k_coarse_slots12(LatView lv, const DT* __restrict__ delta,
                                                       const DT* __restrict__ delta_rf, double* __restrict__ slots,
                                                       const IterCtl* ctl) {
  slots12_body<DT, FULL, AT>(lv, delta, delta_rf, slots, ctl, blockIdx.x);
}

// Batched (per-iteration pass, FULL = false): the sets of every problem.
template <typename DT, typename AT>
__global__ void __launch_bounds__(NT) kb_coarse_slots(const BatchProb* __restrict__ P,
                                                      const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = P[it.prob];
  slots_body<DT, false, AT>(q.lv, (const DT*)q.delta, q.slots_it, q.ctl, it.bx);
}

// Band (lower, column-major: band[c*(bw+1) + k] = A[c+k][c]) of K_aa from the
// base (modes 1-6) and per-iteration (modes 7-q) slots; q modes per set, slots
// of 2q x 2q.
__device__ inline double slot_entry(const double* base, const double* it, int q, int I, int slot, int p, int c) {
  const size_t o = ((size_t)I * NSLOTS + slot) * slot_size(q) + (size_t)p * slot_dim(q) + c;
  return base[o] + it[o];
}

__device__ __forceinline__ void band_from_slots_body(const LatView lv, const double* __restrict__ base,
                                                     const double* __restrict__ it, double* __restrict__ band,
                                                     int bw, const IterCtl* ctl, int bx, int gx) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  const int nm = lv.q;
  const int n = nm * lv.M;
  const size_t total = (size_t)n * (bw + 1);
  for (size_t q = bx * (size_t)blockDim.x + threadIdx.x; q < total;
       q += (size_t)gx * blockDim.x) {
    const int col = (int)(q / (bw + 1)), k = (int)(q % (bw + 1));
    const int row = col + k;
    double v = 0.0;
    if (row < n) {
      const int I = col / nm, m = col % nm;
      const int J = row / nm, l = row % nm;
      const int Ix = I % lv.Mx, Iy = I / lv.Mx, Jx = J % lv.Mx, Jy = J / lv.Mx;
      if (J == I) {
        v = slot_entry(base, it, nm, I, SLOT_SELF, l, m);
        for (int s = SLOT_E; s < NSLOTS; ++s) v += slot_entry(base, it, nm, I, s, l, m);
        // contributions of neighbours that own bars into I
        const int kx[5] = {-1, 1, 0, -1, 1};   // owner offset for E, W, N, NE, NW
        const int ky[5] = {0, 0, -1, -1, -1};
        for (int s = 0; s < 5; ++s) {
          const int Kx = Ix + kx[s], Ky = Iy + ky[s];
          if (Kx < 0 || Kx >= lv.Mx || Ky < 0 || Ky >= lv.My) continue;
          v += slot_entry(base, it, nm, Ky * lv.Mx + Kx, SLOT_E + s, nm + l, nm + m);
        }
      } else {
        const int dx = Jx - Ix, dy = Jy - Iy;
        if (dy == 0 && dx == 1) {
          v = slot_entry(base, it, nm, I, SLOT_E, nm + l, m) + slot_entry(base, it, nm, J, SLOT_W, l, nm + m);
        } else if (dy == 1 && dx == 0) {
          v = slot_entry(base, it, nm, I, SLOT_N, nm + l, m);
        } else if (dy == 1 && dx == 1) {
          v = slot_entry(base, it, nm, I, SLOT_NE, nm + l, m);
        } else if (dy == 1 && dx == -1) {
          v = slot_entry(base, it, nm, I, SLOT_NW, nm + l, m);
        }
      }
    }
    band[q] = v;
  }
}

__global__ void k_band_from_slots(LatView lv, const double* __restrict__ base,
                                  const double* __restrict__ it, double* __restrict__ band, int bw,
                                  const IterCtl* ctl) {
  band_from_slots_body(lv, base, it, band, bw, ctl, blockIdx.x, gridDim.x);
}
__global__ void kb_band_from_slots(const BatchProb* __restrict__ P, const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = P[it.prob];
  band_from_slots_body(q.lv, q.slots_base, q.slots_it, q.band, q.bw, q.ctl, it.bx, it.gx);
}

__global__ void k_band_from_dense(int n, int bw, const double* __restrict__ dense,
                                  double* __restrict__ band) {
  const size_t total = (size_t)n * (bw + 1);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
       q += (size_t)gridDim.x * blockDim.x) {
    const int col = (int)(q / (bw + 1)), k = (int)(q % (bw + 1));
    const int row = col + k;
    band[q] = row < n ? dense[(size_t)row * n + col] : 0.0;
  }
}

__global__ void k_dense_from_band(int n, int bw, const double* __restrict__ band,
                                  double* __restrict__ dense) {
  const size_t total = (size_t)n * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
       q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), c = (int)(q % n);
    const int hi = r > c ? r : c, lo = r > c ? c : r;
    dense[q] = (hi - lo <= bw) ? band[(size_t)lo * (bw + 1) + (hi - lo)] : 0.0;
  }
}

// Jacobi scaling (s_i = D_ii^-1/2), right-hand side b = s P, the solution
// accumulator x = 0, and the modes that take no part: those left out by the
// mode mask (bit m keeps mode m of every set) and those that vanish, D_ii <=
// 1e-300 or <= 1e-28 times the largest diagonal of the set's modes that are
// kept (zero up to rounding).
__device__ __forceinline__ void coarse_diag_body(int n, int bw, const double* __restrict__ band,
                                                 const double* __restrict__ P, double* __restrict__ scale,
                                                 double* __restrict__ b, double* __restrict__ x,
                                                 int* __restrict__ dropped, unsigned mode_mask, int nm,
                                                 const IterCtl* ctl, int bx, int gx) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  for (int i = bx * blockDim.x + threadIdx.x; i < n; i += gx * blockDim.x) {
    const double D = band[(size_t)i * (bw + 1)];
    const int g0 = i - i % nm;
    double dmax = 0.0;
    for (int m = 0; m < nm && g0 + m < n; ++m)
      if ((mode_mask >> m) & 1u) dmax = fmax(dmax, band[(size_t)(g0 + m) * (bw + 1)]);
    const bool drop = !((mode_mask >> (i % nm)) & 1u) || !(D > 1e-300) || !(D > 1e-28 * dmax);
    const double s = drop ? 0.0 : 1.0 / sqrt(D);
    scale[i] = s;
    b[i] = s * P[i];
    x[i] = 0.0;
    dropped[i] = drop ? 1 : 0;
  }
}

__global__ void k_coarse_diag(int n, int bw, const double* __restrict__ band,
                              const double* __restrict__ P, double* __restrict__ scale,
                              double* __restrict__ b, double* __restrict__ x, int* __restrict__ dropped,
                              unsigned mode_mask, int nm, const IterCtl* ctl) {
  coarse_diag_body(n, bw, band, P, scale, b, x, dropped, mode_mask, nm, ctl, blockIdx.x, gridDim.x);
}
__global__ void kb_coarse_diag(const BatchProb* __restrict__ Pb, const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = Pb[it.prob];
  coarse_diag_body(q.n_c, q.bw, q.band, q.P, q.scale, q.b, q.x, q.dropped, q.mode_mask, NMODES, q.ctl, it.bx, it.gx);
}

// Modes that depend on earlier modes of the same set get a = 0.  Sets have
// disjoint supports, so the columns of V can only be dependent within a set:
// the Jacobi-scaled 9 x 9 diagonal block of every set is factored in FP64 in
// mode order, and a mode whose pivot is <= 1e-14 is dropped (the rule of the
// full upper-level system, decided where FP64 resolves it).
template <int Q = NMODES>
__device__ __forceinline__ void set_drops_body(int nsets, int bw, const double* __restrict__ band,
                                               const double* __restrict__ scale, int* __restrict__ dropped,
                                               const IterCtl* ctl, int bx, int gx) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  const int I = bx * blockDim.x + threadIdx.x;
  if (I >= nsets) return;
  constexpr int NMODES = Q;  // modes per set (shadows the 9 of the displacement-controlled form)
  double A[NMODES][NMODES];
  bool dr[NMODES];
#pragma unroll
  for (int m = 0; m < NMODES; ++m) {
    dr[m] = dropped[NMODES * I + m] != 0;
#pragma unroll
    for (int l = 0; l < NMODES; ++l) {
      const int lo = l < m ? l : m, hi = l < m ? m : l;
      const int c = NMODES * I + lo;
      A[m][l] = scale[NMODES * I + m] * band[(size_t)c * (bw + 1) + (hi - lo)] * scale[NMODES * I + l];
    }
  }
#pragma unroll
  for (int m = 0; m < NMODES; ++m) {
    if (dr[m]) continue;
    double piv = A[m][m];
#pragma unroll
    for (int k = 0; k < m; ++k) piv -= A[m][k] * A[m][k];
    if (!(piv > 1e-14)) {
      dr[m] = true;  // its column of L is zero
#pragma unroll
      for (int l = m + 1; l < NMODES; ++l) A[l][m] = 0.0;
      continue;
    }
    const double d = sqrt(piv);
    A[m][m] = d;
#pragma unroll
    for (int l = m + 1; l < NMODES; ++l) {
      if (dr[l]) continue;
      double v = A[l][m];
#pragma unroll
      for (int k = 0; k < m; ++k) v -= A[l][k] * A[m][k];
      A[l][m] = v / d;
    }
  }
#pragma unroll
  for (int m = 0; m < NMODES; ++m) dropped[NMODES * I + m] = dr[m] ? 1 : 0;
}

template <int Q>
__global__ void k_coarse_set_drops(int nsets, int bw, const double* __restrict__ band,
                                   const double* __restrict__ scale, int* __restrict__ dropped,
                                   const IterCtl* ctl) {
  set_drops_body<Q>(nsets, bw, band, scale, dropped, ctl, blockIdx.x, gridDim.x);
}
__global__ void kb_coarse_set_drops(const BatchProb* __restrict__ P, const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = P[it.prob];
  set_drops_body(q.lv.M, q.bw, q.band, q.scale, q.dropped, q.ctl, it.bx, it.gx);
}

// Scaled band in FP64 (column layout for the residual's upper part and row
// layout for its lower part) and the factor's input in row layout, in T.
template <typename T>
__device__ __forceinline__ void scale_band_body(int n, int bw, const double* __restrict__ band,
                                                const double* __restrict__ scale, const int* __restrict__ dropped,
                                                double* __restrict__ sband, double* __restrict__ sbandR,
                                                T* __restrict__ frow, double* __restrict__ b, const IterCtl* ctl,
                                                int bx, int gx) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  const size_t total = (size_t)n * (bw + 1);
  for (size_t q = bx * (size_t)blockDim.x + threadIdx.x; q < total;
       q += (size_t)gx * blockDim.x) {
    const int col = (int)(q / (bw + 1)), k = (int)(q % (bw + 1));
    const int row = col + k;
    double v = 0.0;
    if (row < n) {
      if (k == 0) {
        v = 1.0;
      } else if (!dropped[row] && !dropped[col]) {
        v = scale[row] * band[q] * scale[col];
      }
    }
    sband[q] = v;
    if (row < n) {
      sbandR[(size_t)row * (bw + 1) + k] = v;
      frow[(size_t)row * (bw + 1) + k] = (T)v;
    }
    if (k == 0 && dropped[col]) b[col] = 0.0;
  }
}

template <typename T>
__global__ void k_coarse_scale_band(int n, int bw, const double* __restrict__ band,
                                    const double* __restrict__ scale, const int* __restrict__ dropped,
                                    double* __restrict__ sband, double* __restrict__ sbandR,
                                    T* __restrict__ frow, double* __restrict__ b, const IterCtl* ctl) {
  scale_band_body<T>(n, bw, band, scale, dropped, sband, sbandR, frow, b, ctl, blockIdx.x, gridDim.x);
}
// Batched: the FP32 factor's input (the batched path factors in FP32).
__global__ void kb_coarse_scale_band(const BatchProb* __restrict__ P, const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = P[it.prob];
  scale_band_body<float>(q.n_c, q.bw, q.band, q.scale, q.dropped, q.sband, q.sband + (size_t)q.n_c * (q.bw + 1),
                         q.lrow, q.b, q.ctl, it.bx, it.gx);
}

}  // namespace

int coarse_bw(const LatView& lv) {
  // set I couples to I + Mx + 1 at most (NE neighbour)
  const int reach = (lv.M > 1) ? (lv.Mx + 1 < lv.M - 1 ? lv.Mx + 1 : lv.M - 1) : 0;
  return lv.q * (reach + 1) - 1;
}

size_t coarse_slots_smem(const LatView& lv) {
  const int w = lv.sx < lv.nx ? lv.sx : lv.nx;
  const int h = lv.sy < lv.ny ? lv.sy : lv.ny;
  // interface lists, then the reduction buffer and the CTA totals
  if (lv.q == NMODES_RF)
    return ((size_t)list_caps(w, h).total * LSTRIDE12 + RED_CHUNK * NT + NGEN12_DELTA) * sizeof(double);
  return ((size_t)list_caps(w, h).total * LSTRIDE + RED_CHUNK * NT + NREG + NGEN_FULL) * sizeof(double);
}

cudaError_t launch_coarse_slots(cudaStream_t s, const LatView& lv, const void* delta, bool delta_fp32,
                                bool full, double* slots, const IterCtl* ctl, const void* delta_rf) {
  const size_t smem = coarse_slots_smem(lv);
  if (lv.q == NMODES_RF) {
    if (delta_fp32) {
      const float2 *d = (const float2*)delta, *f = (const float2*)delta_rf;
      if (full) k_coarse_slots12<float2, true, double><<<lv.M, NT, smem, s>>>(lv, d, f, slots, ctl);
      else k_coarse_slots12<float2, false, float><<<lv.M, NT, smem, s>>>(lv, d, f, slots, ctl);
    } else {
      const double2 *d = (const double2*)delta, *f = (const double2*)delta_rf;
      if (full) k_coarse_slots12<double2, true, double><<<lv.M, NT, smem, s>>>(lv, d, f, slots, ctl);
      else k_coarse_slots12<double2, false, double><<<lv.M, NT, smem, s>>>(lv, d, f, slots, ctl);
    }
    return cudaGetLastError();
  }
  if (delta_fp32) {
    if (full) k_coarse_slots<float2, true, double><<<lv.M, NT, smem, s>>>(lv, (const float2*)delta, slots, ctl);
    else k_coarse_slots<float2, false, float><<<lv.M, NT, smem, s>>>(lv, (const float2*)delta, slots, ctl);
  } else {
    if (full) k_coarse_slots<double2, true, double><<<lv.M, NT, smem, s>>>(lv, (const double2*)delta, slots, ctl);
    else k_coarse_slots<double2, false, double><<<lv.M, NT, smem, s>>>(lv, (const double2*)delta, slots, ctl);
  }
  return cudaGetLastError();
}

cudaError_t configure_coarse_assemble(int max_smem) {
  cudaError_t e;
  if ((e = set_max_dynamic_smem(k_coarse_slots12<float2, true, double>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_slots12<float2, false, float>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_slots12<double2, true, double>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_slots12<double2, false, double>, max_smem)) != cudaSuccess) return e;
  e = set_max_dynamic_smem(k_coarse_slots<float2, true, double>, max_smem);
  if (e != cudaSuccess) return e;
  e = set_max_dynamic_smem(k_coarse_slots<float2, false, float>, max_smem);
  if (e != cudaSuccess) return e;
  e = set_max_dynamic_smem(k_coarse_slots<double2, true, double>, max_smem);
  if (e != cudaSuccess) return e;
  e = set_max_dynamic_smem(k_coarse_slots<double2, false, double>, max_smem);
  if (e != cudaSuccess) return e;
  e = set_max_dynamic_smem(kb_coarse_slots<float2, float>, max_smem);
  if (e != cudaSuccess) return e;
  return set_max_dynamic_smem(kb_coarse_slots<double2, double>, max_smem);
}

static int grid_for(size_t total) {
  size_t g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

int coarse_grid_for(size_t n) { return grid_for(n); }
int set_drops_blocks(int nsets) { return (nsets + 127) / 128; }

cudaError_t launch_batch_slots(cudaStream_t s, bool fp32, size_t smem, const BatchProb* P, const BatchItem* it,
                               int n) {
  if (n <= 0) return cudaSuccess;
  if (fp32) kb_coarse_slots<float2, float><<<n, NT, smem, s>>>(P, it);
  else kb_coarse_slots<double2, double><<<n, NT, smem, s>>>(P, it);
  return cudaGetLastError();
}
cudaError_t launch_batch_band(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n) {
  if (n <= 0) return cudaSuccess;
  kb_band_from_slots<<<n, 256, 0, s>>>(P, it);
  return cudaGetLastError();
}
cudaError_t launch_batch_diag(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n) {
  if (n <= 0) return cudaSuccess;
  kb_coarse_diag<<<n, 256, 0, s>>>(P, it);
  return cudaGetLastError();
}
cudaError_t launch_batch_set_drops(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n) {
  if (n <= 0) return cudaSuccess;
  kb_coarse_set_drops<<<n, 128, 0, s>>>(P, it);
  return cudaGetLastError();
}
cudaError_t launch_batch_scale_band(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n) {
  if (n <= 0) return cudaSuccess;
  kb_coarse_scale_band<<<n, 256, 0, s>>>(P, it);
  return cudaGetLastError();
}

cudaError_t launch_coarse_band_from_slots(cudaStream_t s, const LatView& lv, const double* base,
                                          const double* slots, double* band, const IterCtl* ctl) {
  const int bw = coarse_bw(lv);
  const size_t total = (size_t)NMODES * lv.M * (bw + 1);
  k_band_from_slots<<<grid_for(total), 256, 0, s>>>(lv, base, slots, band, bw, ctl);
  return cudaGetLastError();
}

cudaError_t launch_coarse_band_from_dense(cudaStream_t s, int n, int bw, const double* dense,
                                          double* band) {
  k_band_from_dense<<<grid_for((size_t)n * (bw + 1)), 256, 0, s>>>(n, bw, dense, band);
  return cudaGetLastError();
}

cudaError_t launch_coarse_dense_from_band(cudaStream_t s, int n, int bw, const double* band,
                                          double* dense) {
  k_dense_from_band<<<grid_for((size_t)n * n), 256, 0, s>>>(n, bw, band, dense);
  return cudaGetLastError();
}

cudaError_t launch_coarse_scale(cudaStream_t s, int n, int bw, bool fp64, const double* band, const double* P,
                                double* sband, void* frow, double* scale, double* b, double* x, int* dropped,
                                unsigned mode_mask, int nm, const IterCtl* ctl) {
  k_coarse_diag<<<grid_for(n), 256, 0, s>>>(n, bw, band, P, scale, b, x, dropped, mode_mask, nm, ctl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nsets = n / nm;
  if (nm == NMODES_RF)
    k_coarse_set_drops<NMODES_RF><<<(nsets + 127) / 128, 128, 0, s>>>(nsets, bw, band, scale, dropped, ctl);
  else
    k_coarse_set_drops<NMODES><<<(nsets + 127) / 128, 128, 0, s>>>(nsets, bw, band, scale, dropped, ctl);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double* sbandR = sband + (size_t)n * (bw + 1);
  const int g = grid_for((size_t)n * (bw + 1));
  if (fp64)
    k_coarse_scale_band<double><<<g, 256, 0, s>>>(n, bw, band, scale, dropped, sband, sbandR, (double*)frow, b, ctl);
  else
    k_coarse_scale_band<float><<<g, 256, 0, s>>>(n, bw, band, scale, dropped, sband, sbandR, (float*)frow, b, ctl);
  return cudaGetLastError();
}

}  // namespace hms
