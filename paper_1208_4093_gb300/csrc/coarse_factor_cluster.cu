// K4 on a thread-block cluster: the FP32 band Cholesky of Eq. 8's scaled
// matrix (the factor of k_coarse_factor<float> in coarse_solve.cu, same
// result up to summation order) with the work of each 16-column block spread
// over CL CTAs on CL SMs.
//
// The window of band rows (bw + 16 rows) is split by 16-row blocks: block-row
// b lives in the shared memory of CTA b mod CL, which alone updates it.  Step K
// (columns k0 .. k0 + 15):
//   P1  every CTA reads X_K = L_KK^-1 and its drop mask from the CTA that
//       factored block K (distributed shared memory);
//   P2  every CTA forms the panel rows P = A_panel X_K^T of its block-rows and
//       writes them into the panel copy of every CTA;           cluster barrier
//   P3  the CTA that owns block-row K + 1 applies the panel to that diagonal
//       block, and its warp 0 factors and inverts it (look-ahead) while
//   P4  the other warps of all CTAs apply the rank-16 update to their own rows
//       (4 x 4 register tiles, aligned 16-byte read-modify-writes), and
//   P5  block K's columns of L go to global memory, each row by its owner;
//   P6  the band rows entering the window are loaded by their owner.
//                                                               cluster barrier
// Every thread of every CTA passes the same sequence of cluster barriers (the
// loop has the same trip count everywhere and no exit), and the kernel waits
// on nothing else.
#include <cooperative_groups.h>

#include "coarse_common.cuh"
#include "hms_internal.cuh"

namespace hms {
namespace {

namespace cg = cooperative_groups;
using namespace coarse;

constexpr int CL = 4;      // CTAs per cluster
constexpr int FTC = 512;   // threads per CTA
constexpr int MAXRT = 64;  // local row tiles of one step (bw <= 1023)

struct ClLayout {
  int nbr, nls, lda, pstr;
  size_t pc, xb, lb, total;  // float offsets; the window starts at 0
};
__host__ __device__ inline ClLayout cl_layout(int bw) {
  ClLayout L;
  const int W = (bw > NB ? bw : NB) + NB;
  L.nbr = (W + NB - 1) / NB;          // block-rows of the window
  L.nls = (L.nbr + CL - 1) / CL + 1;  // block-row slots per CTA
  L.lda = window_lda(bw);
  L.pstr = ((bw + 7) / 8) * 8 + 8;    // panel rows [k1, rend), tiles read up to 3 past
  L.pc = (size_t)L.nls * NB * L.lda;
  L.xb = L.pc + (size_t)NB * L.pstr;  // X of a diagonal block, two buffers of NB x (NB + 1)
  L.lb = L.xb + 2 * NB * (NB + 1);    // L of a diagonal block, two buffers
  L.total = L.lb + 2 * NB * (NB + 1);
  return L;
}

__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(FTC, 1)
    k_coarse_factor_cl(int n, int bw, const float* __restrict__ lrow, float* __restrict__ lcol,
                       float* __restrict__ dinv, int* __restrict__ dropped, const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;  // the same flag for every CTA: no barrier is passed
  extern __shared__ __align__(16) unsigned char fsraw[];
  float* fs = reinterpret_cast<float*>(fsraw);
  const ClLayout LY = cl_layout(bw);
  const int lda = LY.lda, ldw = bw + 1, pstr = LY.pstr, nbr = LY.nbr, nls = LY.nls;
  float* Win = fs;
  float* Pc = fs + LY.pc;
  float* Xb = fs + LY.xb;
  float* Lb = fs + LY.lb;
  int* sdrop = reinterpret_cast<int*>(fs + LY.total);
  __shared__ unsigned dropblk[2];
  __shared__ float Xcur[NB * (NB + 1)];
  __shared__ unsigned dcur;
  __shared__ int rt_ti[MAXRT + 1], rt_cum[MAXRT + 1], nrt;

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = (n + NB - 1) / NB;
  float* pc_of[CL];
#pragma unroll
  for (int r = 0; r < CL; ++r) pc_of[r] = cluster.map_shared_rank(Pc, r);

  // window row i (its block-row is owned here): columns at position col mod lda
  auto row_ptr = [&](int i) -> float* {
    const int b = i / NB;
    return Win + (size_t)(((b / CL) % nls) * NB + (i % NB)) * lda;
  };
  auto owns = [&](int b) { return b % CL == rank; };

  for (int i = tid; i < n; i += FTC) sdrop[i] = dropped[i];
  for (int q = tid; q < min(n, nbr * NB) * ldw; q += FTC) {
    const int i = q / ldw, kk = q - (q / ldw) * ldw;
    if (owns(i / NB) && kk <= i) row_ptr(i)[(i - kk) % lda] = lrow[(size_t)i * ldw + kk];
  }
  __syncthreads();
  if (rank == 0 && warp == 0) {
    float a[NB];
    const int nbk = min(NB, n);
#pragma unroll
    for (int j = 0; j < NB; ++j) a[j] = (lane < nbk && j <= lane && lane - j <= bw) ? row_ptr(lane)[j] : 0.f;
    factor_diag_block<float>(a, 0, nbk, lane, sdrop, Lb, Xb, dinv, &dropblk[0]);
  }
  cluster.sync();

  for (int K = 0; K < nblk; ++K) {
    const int owner = K % CL, buf = K & 1;
    const int k0 = K * NB, k1 = min(k0 + NB, n), nbk = k1 - k0;
    const int rend = min(n, k1 + bw), np = rend - k1;
    // ---- P1: X_K and its drop mask from the CTA that factored block K ----
    {
      const float* xr = cluster.map_shared_rank(Xb + buf * NB * (NB + 1), owner);
      for (int q = tid; q < NB * (NB + 1); q += FTC) Xcur[q] = xr[q];
      if (tid == 0) dcur = *cluster.map_shared_rank(&dropblk[buf], owner);
    }
    __syncthreads();
    // ---- P2: panel rows of the local block-rows in [k1, rend), 1 row x 4 columns per thread ----
    {
      const int bfirst = K + 1, blast = (rend - 1) / NB;
      int b0 = bfirst + ((rank - bfirst % CL) % CL + CL) % CL;  // first local block-row >= K + 1
      const int nlocal = (np > 0 && b0 <= blast) ? (blast - b0) / CL + 1 : 0;
      const int ck0 = k0 % lda;
      for (int q = tid; q < nlocal * NB * (NB / 4); q += FTC) {
        const int lb = q / (NB * (NB / 4)), rq = q % (NB * (NB / 4));
        const int r16 = rq >> 2, cq = rq & 3;
        const int i = (b0 + lb * CL) * NB + r16;
        if (i >= rend) continue;
        const float* ar = row_ptr(i);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int cp = 0; cp < NB; ++cp) {
          const int kk = i - (k0 + cp);
          const int p = ck0 + cp;
          const float av = (kk <= bw) ? ar[p >= lda ? p - lda : p] : 0.f;
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[v] = fmaf(av, Xcur[(4 * cq + v) * (NB + 1) + cp], acc[v]);
        }
        const int il = i - k1;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int c = 4 * cq + v;
          const float val = (c < nbk && !((dcur >> c) & 1u)) ? acc[v] : 0.f;
#pragma unroll
          for (int r = 0; r < CL; ++r) pc_of[r][c * pstr + il] = val;
        }
      }
    }
    cluster.sync();  // the whole panel in every CTA; block K's X no longer read
    const int nown = (K + 1) % CL;
    const bool next_here = rank == nown && K + 1 < nblk;
    const int nbk2 = (K + 1 < nblk) ? min(NB, n - k1) : 0;
    if (next_here) {
      // ---- P3a: rank-16 update of diagonal block K + 1 ----
      const int ck1 = k1 % lda;
      for (int q = tid; q < NB * NB; q += FTC) {
        const int l = q / NB, j = q - l * NB;
        if (l < nbk2 && j <= l && l < np && l - j <= bw) {
          float v = 0.f;
#pragma unroll
          for (int c = 0; c < NB; ++c) v = fmaf(Pc[c * pstr + l], Pc[c * pstr + j], v);
          const int p = ck1 + j;
          row_ptr(k1 + l)[p >= lda ? p - lda : p] -= v;
        }
      }
      __syncthreads();
    }
    // local row tiles of the trailing update: 4-row tiles of the local block-rows >= K + 2
    if (tid == 0) {
      int cnt = 0, cum = 0;
      const int blast = (rend - 1) / NB;
      for (int b = K + 2; b <= blast && np > 0; ++b) {
        if (!owns(b)) continue;
        for (int u = 0; u < NB / 4; ++u) {
          const int row0 = b * NB + 4 * u;
          if (row0 >= rend || cnt >= MAXRT) break;
          const int ti = (row0 - k1) / 4;
          rt_ti[cnt] = ti;
          rt_cum[cnt] = cum;
          cum += ti + 1;
          ++cnt;
        }
      }
      rt_cum[cnt] = cum;
      nrt = cnt;
    }
    __syncthreads();
    const bool diag_warp = next_here && warp == 0;
    const bool light_warp = next_here && warp != 0 && (warp & 3) == 0;  // shares warp 0's scheduler
    if (diag_warp) {
      // ---- P3b: factor and invert diagonal block K + 1 ----
      float a[NB];
      const float* ar = row_ptr(min(k1 + lane, n - 1));
      const int ck1 = k1 % lda;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int p = ck1 + j;
        a[j] = (lane < nbk2 && j <= lane && lane - j <= bw) ? ar[p >= lda ? p - lda : p] : 0.f;
      }
      factor_diag_block<float>(a, k1, nbk2, lane, sdrop, Lb + (buf ^ 1) * NB * (NB + 1),
                               Xb + (buf ^ 1) * NB * (NB + 1), dinv, &dropblk[buf ^ 1]);
    } else if (!light_warp) {
      // ---- P4: trailing update of the local rows ----
      const int wi = next_here ? warp - 1 - (warp >> 2) : warp;
      const int nwi = next_here ? FTC / 32 - FTC / 128 : FTC / 32;
      const int total = rt_cum[nrt];
      for (int q = wi * 32 + lane; q < total; q += nwi * 32) {
        int k = 0;
        while (k + 1 < nrt && rt_cum[k + 1] <= q) ++k;
        const int ti = rt_ti[k], tj = q - rt_cum[k];
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          const float* pc = Pc + c * pstr;
          float ri[4], rj[4];
          ld4(pc + 4 * ti, ri);
          ld4(pc + 4 * tj, rj);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(ri[u], rj[v], acc[u][v]);
        }
        // (i, k1 + 4 tj .. + 3) is one aligned 16-byte word of row i; entries
        // right of the diagonal in a diagonal tile land on unused positions
        const int pj = (k1 + 4 * tj) % lda;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = k1 + 4 * ti + u;
          if (i >= rend) continue;
          float* w4 = row_ptr(i) + pj;
          float old[4];
          ld4(w4, old);
          st4(w4, old[0] - acc[u][0], old[1] - acc[u][1], old[2] - acc[u][2], old[3] - acc[u][3]);
        }
      }
    }
    if (!diag_warp) {
      // ---- P5: block K's columns of L, each row by its owner ----
      const int wl = light_warp ? (warp >> 2) - 1 : (next_here ? warp - 1 - (warp >> 2) : warp);
      const int nwl = light_warp ? FTC / 128 - 1 : (next_here ? FTC / 32 - FTC / 128 : FTC / 32);
      const bool lw_role = !next_here || light_warp;  // who writes: the light warps where warp 0 is busy
      if (lw_role) {
        for (int q = wl * 32 + lane; q < nbk * ldw; q += nwl * 32) {
          const int cl = q / ldw, kk = q - cl * ldw;
          const int c = k0 + cl, i = c + kk;
          float v = 0.f;
          bool mine = false;
          if (i < k1) {
            mine = rank == owner;
            if (mine) v = Lb[buf * NB * (NB + 1) + (i - k0) * (NB + 1) + cl];
          } else if (i < rend) {
            mine = owns(i / NB);
            if (mine) v = Pc[cl * pstr + (i - k1)];
          } else {
            mine = rank == owner;  // past the matrix end: zero
          }
          if (mine) lcol[(size_t)c * ldw + kk] = v;
        }
        // ---- P6: the band rows entering the window (block-row K + nbr) ----
        const int be = K + nbr;
        if (owns(be) && be * NB < n) {
          for (int q = wl * 32 + lane; q < NB * ldw; q += nwl * 32) {
            const int r16 = q / ldw, kk = q - r16 * ldw;
            const int i = be * NB + r16;
            if (i < n && kk <= i) row_ptr(i)[(i - kk) % lda] = lrow[(size_t)i * ldw + kk];
          }
        }
      }
    }
    cluster.sync();  // block K + 1's X ready, window updated, entering rows in place
  }
  for (int i = tid; i < n; i += FTC)
    if (owns(i / NB)) dropped[i] = sdrop[i];
}

}  // namespace

size_t coarse_factor_cl_smem_bytes(int n, int bw) {
  if (bw > 1023) return (size_t)1 << 30;
  return cl_layout(bw).total * sizeof(float) + (size_t)n * sizeof(int);
}

cudaError_t configure_coarse_factor_cl(int max_smem) { return set_max_dynamic_smem(k_coarse_factor_cl, max_smem); }

cudaError_t launch_coarse_factor_cl(cudaStream_t s, int n, int bw, const void* lrow, void* lcol, void* dinv,
                                    int* dropped, const IterCtl* ctl) {
  k_coarse_factor_cl<<<CL, FTC, coarse_factor_cl_smem_bytes(n, bw), s>>>(n, bw, (const float*)lrow, (float*)lcol,
                                                                         (float*)dinv, dropped, ctl);
  return cudaGetLastError();
}

}  // namespace hms
