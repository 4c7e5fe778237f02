// K2: displacement-controlled local relaxation of every set (Eqs. 11-13) and
// the upper-level force P = V^T r (Eq. 7).
//
// Eq. 12 fixes the outer displacements at their old values and solves
//   k^Inner u^RD = p^Inner - k^Outer u^Outer-old.
// Subtracting k^Inner u^Inner-old from both sides gives the increment of
// Eq. 13 directly from the global residual:
//   k^Inner (u^RD - u^old) = p^Inner - k^Outer u^Outer-old - k^Inner u^Inner-old = r_I,
// so delta_I = (k^Inner_I)^-1 r_I, all sets from the same u (every set relaxes
// against its neighbours' old displacements).  With an extended relaxation
// region (Sec. 2.2; LatView::ov > 0) the same solve runs on the set's tile
// grown by ov nodes and delta is kept on the set's own nodes.
//
// One CTA per set.  The set's block-bidiagonal factor (setup.cu) is a stream
// of matrices Linv_0, B_1, Linv_1, ..., consumed in order by the forward
// substitution and, from the copy stored by columns, in reverse order by the
// back substitution:
//   forward  y_j = Linv_j (r_j - B_j y_{j-1})
//   backward x_j = Linv_j^T (y_j - B_{j+1}^T x_{j+1})
// so both passes are products of packed rows with a vector.  Each matrix is
// staged in shared memory by a 1-D bulk copy (cp.async.bulk, completion on an
// mbarrier), three slots deep so two matrices stream in while one is applied
// (with one copy per matrix a step ends in the only barrier it has);
// a B step's vector (r_j forward, y_{j-1} backward) comes in the same
// transaction.  Rows r and nb-1-r of a matrix go to a group of G threads as
// one combined index range of almost constant length (nb+1 for the triangles,
// about nb+7 for the B blocks), so every lane of a warp runs the same number
// of FMAs.  The solve runs in T = double (FP64 path) or T = float (mixed path,
// FP32 factor), with G = 4 threads per row pair either way.  After the back
// substitution the nine sums of P_I = V_I^T r_I are formed in FP64 from r and
// the delta just written, node by node.
//
// The copies are issued by one more warp (the producer, threads NT .. NT+31),
// which takes no part in the products: issuing a copy (fences, the expected
// byte count, the copy instructions) would otherwise delay one compute warp,
// and with it the whole step, at every matrix.
//
// The compute CTA size NT (64, 128 or 256 threads) and, in FP64, the copies per matrix
// NC (1, or 2: the outer and the inner row pairs apart, half the shared memory
// per slot) are launch choices: NT / G row pairs are worked on at once, so 32
// x 32-node sets (32 pairs) fill a CTA of 128 threads and 64 x 64-node sets
// one of 256.  Every row's sum and every P sum is formed in the same order
// whatever NT and NC are (the P sums over 256 virtual lanes), so the results
// are bitwise the same for every choice, and the problem setup may pick them
// by timing (relax_threads = 0).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "hms_internal.cuh"
#include "ptx.cuh"

namespace hms {
namespace {

constexpr int VL = 256;  // virtual lanes of the P sums (8 virtual warps)

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

constexpr int NSLOT = 3;  // matrices staged in shared memory (two in flight while one is applied)

struct RelaxSmem {
  size_t slot_elems, vec_off, vec_elems, ycur_off, z_off, w_off, x_off, total_elems;
};

// Row stride of the y scratch: nb rounded up to 4 entries, so that every row
// starts on 16 bytes (the bulk copies' rule).
__host__ __device__ inline int y_row(int nb) { return (nb + 3) / 4 * 4; }

// Row offsets within a matrix of each kind, and the storage size (padded).
__host__ __device__ inline long long kind_row_off(int kind, int nb, int r) {
  switch (kind) {
    case 0: return linv_row_off(r);
    case 1: return b_row_off(nb, r);
    case 2: return lt_row_off(nb, r);
    default: return bt_row_off(nb, r);
  }
}
__host__ __device__ inline long long kind_size(int kind, int nb) {
  return (kind == 0 || kind == 2) ? linv_size(nb) : b_size(nb);
}

// Two copies per matrix (NC = 2): the rows of the pairs (r, nb-1-r) with
// r < r1 ("outer", rows [0, r1) and [nb-r1, nb)) and those with r >= r1
// ("inner", rows [r1, nb-r1)), about half the matrix each, so that a CTA
// needs only half the shared memory per slot.  r1 is the value nearest nb/4
// at which every kind's row offsets at r1 and nb-r1 start on 16 bytes (the
// bulk copies' rule); 0 if there is none.
template <typename T>
__host__ __device__ inline int chunk_r1(int nb) {
  const long long a = 16 / sizeof(T);
  for (int d = 0; d <= 8; ++d)
    for (int sgn = 0; sgn < 2; ++sgn) {
      const int r1 = nb / 4 + (sgn ? -d : d);
      if (r1 < 1 || 2 * r1 >= nb) continue;
      bool ok = true;
      for (int kind = 0; kind < 4 && ok; ++kind)
        ok = kind_row_off(kind, nb, r1) % a == 0 && kind_row_off(kind, nb, nb - r1) % a == 0;
      if (ok) return r1;
    }
  return 0;
}
// elements of chunk c (0 outer, 1 inner) of a matrix of the kind
__host__ __device__ inline long long chunk_elems(int kind, int nb, int r1, int c) {
  const long long lo = kind_row_off(kind, nb, r1), hi = kind_row_off(kind, nb, nb - r1);
  return c == 0 ? lo + (kind_size(kind, nb) - hi) : hi - lo;
}

template <typename T, int NC = 1>
__host__ __device__ inline RelaxSmem relax_layout(int nb) {
  RelaxSmem L;
  long long ls = linv_size(nb), bs = b_size(nb);
  L.slot_elems = (size_t)(ls > bs ? ls : bs);
  if (NC == 2) {
    const int r1 = chunk_r1<T>(nb);
    long long m = 0;
    for (int kind = 0; kind < 4; ++kind)
      for (int c = 0; c < 2; ++c) {
        const long long e = chunk_elems(kind, nb, r1, c);
        m = e > m ? e : m;
      }
    L.slot_elems = (size_t)m;
  }
  const size_t a = 16 / sizeof(T);  // keep every region 16-byte aligned
  auto up = [a](size_t n) { return (n + a - 1) / a * a; };
  // per slot, the vector a B step reads besides the product: r_j (FP64) in the
  // forward pass, y_{j-1} in the backward pass; staged with the matrix
  L.vec_off = up(NSLOT * L.slot_elems);
  {
    const size_t rb = (size_t)nb * sizeof(double), yb = (size_t)y_row(nb) * sizeof(T);  // r_j, y_{j-1}
    L.vec_elems = up(((rb > yb ? rb : yb) + sizeof(T) - 1) / sizeof(T));
  }
  L.ycur_off = up(L.vec_off + NSLOT * L.vec_elems);
  L.z_off = up(L.ycur_off + nb);
  L.w_off = up(L.z_off + nb);
  L.x_off = up(L.w_off + nb);
  L.total_elems = up(L.x_off + nb);
  return L;
}

// Dot products of rows ra and rb (ra < rb) of a packed matrix M with v.  Row
// x holds v-indices lo_x .. lo_x + len_x - 1, stored from M + off_x.  The G
// threads of a group (g = 0..G-1) walk the combined index t = 0..lenA+lenB-1
// with stride G, in CH interleaved chains of FMAs.  Returns the sum of row A
// in the group's even threads and of row B in its odd threads.
template <typename T, int G, int CH>
__device__ inline void pair_dot(const T* __restrict__ pA, int loA, int lenA, const T* __restrict__ pB, int loB,
                                int lenB, const T* __restrict__ v, int g, T& out) {
  static_assert(CH == 1 || CH == 2, "one or two chains per thread");
  const int len = lenA + lenB;
  T a[CH], b[CH];
#pragma unroll
  for (int q = 0; q < CH; ++q) a[q] = b[q] = T(0);
  // The combined index t (row A's entries, then row B's) is walked from g with
  // stride G, entry t going to chain ((t - g) / G) mod CH.
  if constexpr (CH == 1) {
    // FP64: one walk with the row chosen per entry.  Every lane of a warp then
    // runs the same number of FMAs (len is nearly the same for every pair),
    // which matters where a warp's FMA holds the FP64 pipe whatever its
    // active lanes.  The walk keeps one running sum and, where its index
    // passes lenA, moves that sum to row A's and starts row B's from zero (so
    // no select sits between two FMAs of the chain); the next entry's two
    // operands are loaded before this entry's FMA, so the shared-memory
    // latency overlaps the chain.
    if (g < len) {
      bool inA = g < lenA;
      const T* mb = inA ? pA : pB - lenA;  // entry t of the walk: mb[t] * xb[t]
      const T* xb = inA ? v + loA : v + (loB - lenA);
      T m = mb[g], x = xb[g];
      T acc = T(0), accA = T(0);
      for (int t = g; t < len; t += G) {
        const int tn = t + G;
        const bool cross = inA && tn >= lenA;  // entry tn is this thread's first of row B
        if (cross) {
          mb = pB - lenA;
          xb = v + (loB - lenA);
        }
        T mn = T(0), xn = T(0);
        if (tn < len) {
          mn = mb[tn];
          xn = xb[tn];
        }
        acc = fma(m, x, acc);
        if (cross) {
          accA = acc;
          acc = T(0);
          inA = false;
        }
        m = mn;
        x = xn;
      }
      if (inA) {
        a[0] = acc;
      } else {
        a[0] = accA;
        b[0] = acc;
      }
    }
  } else {
    // FP32: row A's part and row B's part as two plain loops (no per-entry
    // choice of row: the index arithmetic, not the FMAs, bound the one
    // walk), each entry landing in the same chain and order as in one walk.
    const T* va = v + loA;
    int t = g;
    for (; t + G < lenA; t += 2 * G) {
      a[0] = fma(pA[t], va[t], a[0]);
      a[1] = fma(pA[t + G], va[t + G], a[1]);
    }
    if (t < lenA) a[0] = fma(pA[t], va[t], a[0]);
    // row B from the first t >= lenA of this thread's walk; its chain is q0
    const int t0 = lenA + ((g - lenA) & (G - 1));
    const int q0 = ((t0 - g) / G) & 1;
    const T* mb = pB - lenA;  // indexed by the combined t >= lenA
    const T* vb = v + (loB - lenA);
    T b0 = T(0), b1 = T(0);  // the chains in walk order: q0, then the other
    for (t = t0; t + G < len; t += 2 * G) {
      b0 = fma(mb[t], vb[t], b0);
      b1 = fma(mb[t + G], vb[t + G], b1);
    }
    if (t < len) b0 = fma(mb[t], vb[t], b0);
    b[0] = q0 ? b1 : b0;
    b[CH - 1] = q0 ? b0 : b1;
  }
  T sa = a[0], sb = b[0];
#pragma unroll
  for (int q = 1; q < CH; ++q) sa += a[q], sb += b[q];
  // joint reduction over the group: after the first exchange even threads
  // hold partial sums of row A and odd threads of row B
  const bool odd = (g & 1) != 0;
  T s = odd ? sb : sa;
  s += __shfl_xor_sync(0xffffffffu, odd ? sa : sb, 1);
#pragma unroll
  for (int m = 2; m < G; m <<= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  out = s;  // row A in threads g = 0, 2, ..., row B in g = 1, 3, ...
}

// The four kinds of matrix rows: lowest v-index, entry count and storage offset.
enum RowKind { ROW_LINV = 0, ROW_B, ROW_LT, ROW_BT };
template <int K>
__device__ inline void row_shape(int nb, int r, int& lo, int& len, long long& off) {
  if (K == ROW_LINV) {
    lo = 0; len = r + 1; off = linv_row_off(r);
  } else if (K == ROW_B) {
    lo = b_lo(r); len = nb - lo; off = b_row_off(nb, r);
  } else if (K == ROW_LT) {
    lo = r; len = nb - r; off = lt_row_off(nb, r);
  } else {
    lo = 0; len = bt_hi(nb, r) + 1; off = bt_row_off(nb, r);
  }
}

// out(r, sum, pre) for every row r of the matrix: groups of G threads take
// the row pairs (r, nb-1-r); thread 0 of a group handles row r and thread 1
// row nb-1-r.  pre = fetch(r) is loaded before the products so that its
// latency hides behind them.
//
// Only the pairs [pa, pb) are taken; the slot M holds the rows from storage
// offset base_lo on (rows r < cut) and base_hi on (rows >= cut), i.e. a row's
// place in M is its storage offset minus its base.
template <int NT, typename T, int G, int CH, int K, class Fetch, class Out>
__device__ inline void rows_times(const T* M, const T* v, int nb, int pa, int pb, long long base_lo, int cut,
                                  long long base_hi, Fetch fetch, Out out) {
  const int g = threadIdx.x % G;
  for (int base = pa; base < pb; base += NT / G) {
    const int pq = base + (int)threadIdx.x / G;
    if (base + (int)(threadIdx.x & ~31u) / G >= pb) break;  // the whole warp is past the last pair
    const bool active = pq < pb;
    const int ra = active ? pq : pa, rb = nb - 1 - ra;
    int loA, lenA, loB, lenB;
    long long offA, offB;
    row_shape<K>(nb, ra, loA, lenA, offA);
    row_shape<K>(nb, rb, loB, lenB, offB);
    offA -= ra < cut ? base_lo : base_hi;
    offB -= rb < cut ? base_lo : base_hi;
    if (!active) lenA = lenB = 0;
    const int myrow = (g & 1) ? rb : ra;
    const bool mine = active && g < 2;
    const T pre = mine ? fetch(myrow) : T(0);
    T s;
    pair_dot<T, G, CH>(M + offA, loA, lenA, M + offB, loB, lenB, v, g, s);
    if (mine) out(myrow, s, pre);
  }
}

// Entries of one set's slice of the y scratch (the widest, tallest relaxation region).
__host__ __device__ inline long long y_stride(const LatView& lv) {
  return (long long)y_row(2 * region_w_max(lv)) * region_h_max(lv);
}

// The kernel body for set I.
template <typename T, int NT, int NC>
__device__ __forceinline__ void relax_body(const LatView lv, const long long* __restrict__ set_off,
                                           const T* __restrict__ fac, const double2* __restrict__ r,
                                           T* __restrict__ delta, double* __restrict__ P, T* __restrict__ yglob,
                                           long long ystride, const IterCtl* ctl, int* err, int I, int wait0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint64_t bars[NSLOT];
  __shared__ double pred[(VL / 32) * NMODES];
  __shared__ int abort_flag;
  if (ctl && *(volatile const int*)&ctl->done) return;

  using T2 = typename Vec2<T>::type;
  const int tid = threadIdx.x, lane = tid & 31;
  const bool producer = tid >= NT;  // the last warp issues the copies
  const int Ix = I % lv.Mx, Iy = I / lv.Mx;
  const int i0 = Ix * lv.sx, j0 = Iy * lv.sy;  // the set (its P sums)
  const int w = min(lv.sx, lv.nx - i0), h = min(lv.sy, lv.ny - j0);
  // the relaxation region the solve runs on (the set itself without overlap);
  // delta is kept on the set's own nodes
  const Region RG = relax_region(lv, I);
  const int ri0 = RG.i0, rj0 = RG.j0, rh = RG.h;
  const int nb = 2 * RG.w;
  const int keep_lo = 2 * (i0 - ri0), keep_hi = keep_lo + 2 * w;  // the set's DOFs within a region row
  const RelaxSmem LY = relax_layout<T, NC>(nb);
  const int r1 = NC == 2 ? chunk_r1<T>(nb) : 0;
  T* sm = reinterpret_cast<T*>(smraw);
  T* ycur = sm + LY.ycur_off;  // the latest y_j of the forward pass
  T* zbuf = sm + LY.z_off;
  T* wbuf = sm + LY.w_off;
  T* xbuf = sm + LY.x_off;
  T* yg = yglob + (size_t)I * ystride;  // all y_j, read back by the backward pass
  const T* fset = fac + set_off[I];
  const T* fset_t = fset + set_factor_size(nb, rh);  // the copy stored by columns
  const double* rg = reinterpret_cast<const double*>(r);
  const int nmat = 2 * rh - 1;
  const int nops = 2 * nmat * NC;  // one op per matrix copy (NC per matrix)

  auto mat_of_op = [&](int o) {
    const int m = o / NC;
    return m < nmat ? m : 2 * nmat - 1 - m;
  };
  auto kind_of_op = [&](int o) {
    const bool fwd = o / NC < nmat;
    return (mat_of_op(o) & 1) ? (fwd ? 1 : 3) : (fwd ? 0 : 2);
  };
  const int nbr = y_row(nb);
  int issued = 0;  // ops whose copies the producer has issued (producer thread only)
  auto issue = [&](int o) {
    ++issued;
    const int k = mat_of_op(o);
    const int kind = kind_of_op(o);
    const bool fwd = o / NC < nmat;
    uint64_t* bar = &bars[o % NSLOT];
    const T* src = (fwd ? fset : fset_t) + mat_off(nb, k);
    T* dst = sm + (size_t)(o % NSLOT) * LY.slot_elems;
    // a B step's vector: r_j (forward; 16 bytes per node) or y_{j-1} (backward; rows of nbr entries)
    const int jv = (k + 1) / 2;
    const void* vsrc = fwd ? (const void*)(rg + 2 * ((size_t)(rj0 + jv) * lv.nx + ri0))
                           : (const void*)(yg + (size_t)(jv - 1) * nbr);
    const uint32_t vbytes = (k & 1) ? (uint32_t)(fwd ? nb * sizeof(double) : nbr * sizeof(T)) : 0u;
    T* vdst = sm + LY.vec_off + (size_t)(o % NSLOT) * LY.vec_elems;
    fence_proxy_async_smem();
    // y_{j-1} was stored by this CTA's threads in the forward pass (ordered
    // before this thread by the step barriers)
    if (!fwd && (k & 1)) fence_proxy_async_global();
    if (NC == 1) {
      const uint32_t bytes = (uint32_t)(kind_size(kind, nb) * sizeof(T));
      mbar_arrive_expect_tx(bar, bytes + vbytes);
      bulk_g2s(dst, src, bytes, bar);
    } else {
      const long long lo = kind_row_off(kind, nb, r1), hi = kind_row_off(kind, nb, nb - r1);
      if (o % NC == 0) {
        // outer rows: [0, lo) and [hi, size) one after the other
        const uint32_t b0 = (uint32_t)(lo * sizeof(T)), b1 = (uint32_t)((kind_size(kind, nb) - hi) * sizeof(T));
        mbar_arrive_expect_tx(bar, b0 + b1 + vbytes);
        bulk_g2s(dst, src, b0, bar);
        bulk_g2s(dst + lo, src + hi, b1, bar);
      } else {
        const uint32_t b = (uint32_t)((hi - lo) * sizeof(T));
        mbar_arrive_expect_tx(bar, b + vbytes);
        bulk_g2s(dst, src + lo, b, bar);
      }
    }
    if (vbytes) bulk_g2s(vdst, vsrc, vbytes, bar);
  };
  // pair range and slot bases of op o (see rows_times)
  int pa = 0, pb = nb / 2, cut = nb;
  long long base_lo = 0, base_hi = 0;
  auto chunk_of = [&](int o) {
    if (NC == 1) return;
    const int kind = kind_of_op(o);
    const long long lo = kind_row_off(kind, nb, r1), hi = kind_row_off(kind, nb, nb - r1);
    if (o % NC == 0) {
      pa = 0, pb = r1, cut = r1, base_lo = 0, base_hi = hi - lo;
    } else {
      pa = r1, pb = nb / 2, cut = nb, base_lo = lo, base_hi = 0;
    }
  };

  if (tid == 0) {
    abort_flag = 0;
    for (int k = 0; k < NSLOT; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == NT)
    for (int o = 0; o < NSLOT - 1 && o < nops; ++o) issue(o);
  // z = r_0
  const size_t rowbase0 = 2 * ((size_t)rj0 * lv.nx + ri0);
  if (!producer)
    for (int t = tid; t < nb; t += NT) zbuf[t] = (T)rg[rowbase0 + t];
  if (NC == 1) __syncthreads();  // z before op 0 reads it (two copies: op 0's own barrier)

  const double2 rep = lv.rep[I];

  int o_stop = 0;  // the op at which an abort left the loop
  for (int o = 0; o < nops; ++o) {
    o_stop = o;
    const int k = mat_of_op(o);
    const bool is_b = (k & 1) != 0;
    const int j = is_b ? (k + 1) / 2 : k / 2;
    const bool last_copy = (o % NC) == NC - 1;  // the matrix's outputs are complete after it
    // the first wait may be given a shorter bound (tests of the timeout path)
    const uint32_t tries = (o == 0 && wait0 >= 0) ? (uint32_t)wait0 : MBAR_WAIT_TRIES;
    const bool late = !producer && !mbar_wait_bounded(&bars[o % NSLOT], (uint32_t)((o / NSLOT) & 1), tries);
    if (NC != 1) {
      // after the first copy of a matrix there is no end-of-op barrier: this
      // one frees its slot (and decides an abort the same way in every thread)
      if (late) abort_flag = 1;
      __syncthreads();
      if (abort_flag) break;
    }
    // The slot of op o - 1 is free (one copy per matrix: since the barrier
    // that ended op o - 1): stream op o + NSLOT - 1 into it.  With one copy,
    // a wait that ran out is voted on at the end of the op, so every thread
    // leaves the loop there together.
    if (producer) {
      if (tid == NT && o + NSLOT - 1 < nops) issue(o + NSLOT - 1);
      if (NC == 1) {
        if (__syncthreads_or(0)) {
          abort_flag = 1;
          break;
        }
      } else if (last_copy) {
        __syncthreads();
      }
      continue;
    }
    const T* M = sm + (size_t)(o % NSLOT) * LY.slot_elems;
    const T* vstage = sm + LY.vec_off + (size_t)(o % NSLOT) * LY.vec_elems;
    chunk_of(o);
    // 4 threads per row pair keep two warps per SMSP issuing; FP64 FMAs are
    // slow enough that one chain per thread has no stall, FP32 ones want two
    constexpr int G = 4, CH = sizeof(T) == 8 ? 1 : 2;
    if (o / NC < nmat) {
      // ---------------- forward ----------------
      if (is_b) {
        // z = r_j - B_j y_{j-1} (r_j staged with B_j)
        const double* rj = reinterpret_cast<const double*>(vstage);
        rows_times<NT, T, G, CH, ROW_B>(
            M, ycur, nb, pa, pb, base_lo, cut, base_hi, [&](int row) { return (T)rj[row]; },
            [&](int row, T s, T pre) { zbuf[row] = pre - s; });
      } else {
        // y_j = Linv_j z
        T* yj = yg + (size_t)j * nbr;
        rows_times<NT, T, G, CH, ROW_LINV>(
            M, zbuf, nb, pa, pb, base_lo, cut, base_hi, [](int) { return T(0); },
            [&](int row, T s, T) {
              ycur[row] = s;
              yj[row] = s;
            });
      }
    } else {
      // ---------------- backward ----------------
      if (!is_b) {
        // x_j = Linv_j^T w  (w = y_{h-1} for the last row)
        const T* wv = (j == rh - 1) ? ycur : wbuf;
        const size_t rowbase = 2 * ((size_t)(rj0 + j) * lv.nx + ri0);
        const bool keep_row = rj0 + j >= j0 && rj0 + j < j0 + h;
        rows_times<NT, T, G, CH, ROW_LT>(
            M, wv, nb, pa, pb, base_lo, cut, base_hi, [](int) { return T(0); },
            [&](int row, T s, T) {
              xbuf[row] = s;
              if (keep_row && row >= keep_lo && row < keep_hi) delta[rowbase + row] = s;
            });
      } else {
        // w = y_{j-1} - B_j^T x_j (y_{j-1} staged with B_j^T)
        const T* yp = vstage;
        rows_times<NT, T, G, CH, ROW_BT>(
            M, xbuf, nb, pa, pb, base_lo, cut, base_hi, [&](int row) { return yp[row]; },
            [&](int row, T s, T pre) { wbuf[row] = pre - s; });
      }
    }
    if (NC == 1) {
      if (__syncthreads_or(late)) {
        abort_flag = 1;
        break;
      }
    } else if (last_copy) {
      __syncthreads();
    }
  }
  if (abort_flag) {
    // Let the copies still in flight land before the CTA exits: every thread
    // left the loop at op o_stop, whose wait (or an earlier one) gave up, and
    // the ops before it completed, so the ones in flight are o_stop ..
    // issued - 1, one per slot.  The producer waits for exactly those phases.
    if (tid == NT) {
      for (int k = o_stop; k < issued; ++k) mbar_wait_bounded(&bars[k % NSLOT], (uint32_t)((k / NSLOT) & 1));
      atomicOr(err, (int)DEVERR_TIMEOUT);
    }
    return;
  }
  // P = V^T r (Eq. 7) from r and the delta just written, node by node:
  // virtual lane v sums nodes v, v + VL, ...; each virtual warp's 32 lanes go
  // through one shuffle tree, and the 8 virtual warps are added in order.
  // Modes 1-9 of set I at P[q I + m] (q = 9, or 12 with the force-controlled
  // modes); no P (the force-controlled relaxation's solve) with P = nullptr.
  if (P == nullptr) return;
  __syncthreads();
  const T2* d2 = reinterpret_cast<const T2*>(delta);
  for (int vbase = 0; vbase < VL && !producer; vbase += NT) {
    const int v = vbase + tid;
    if (v >= VL) break;  // whole warps (VL is a multiple of 32)
    double pacc[NMODES];
#pragma unroll
    for (int m = 0; m < NMODES; ++m) pacc[m] = 0.0;
    for (int node = v; node < w * h; node += VL) {
      const int jj = node / w, il = node - jj * w;
      const int j = j0 + jj;
      const size_t nidx = (size_t)j * lv.nx + i0 + il;
      const double2 rv = r[nidx];
      const T2 dv = d2[nidx];
      const double xi = fma(lv.L, (double)(i0 + il) + 0.5 * (double)(j & 1), -rep.x);
      const double eta = fma(lv.L * SQ3_2, (double)j, -rep.y);
      const double dr = fma((double)dv.x, rv.x, (double)dv.y * rv.y);
      pacc[0] += rv.x;
      pacc[1] += rv.y;
      pacc[2] = fma(xi, rv.x, pacc[2]);
      pacc[3] = fma(eta, rv.x, pacc[3]);
      pacc[4] = fma(xi, rv.y, pacc[4]);
      pacc[5] = fma(eta, rv.y, pacc[5]);
      pacc[6] += dr;
      pacc[7] = fma(xi, dr, pacc[7]);
      pacc[8] = fma(eta, dr, pacc[8]);
    }
#pragma unroll
    for (int m = 0; m < NMODES; ++m) {
      const double sm2 = warp_sum_d(pacc[m]);
      if (lane == 0) pred[(v >> 5) * NMODES + m] = sm2;
    }
  }
  __syncthreads();
  if (tid < NMODES) {
    double sum = 0.0;
    for (int ww = 0; ww < VL / 32; ++ww) sum += pred[ww * NMODES + tid];
    P[(size_t)lv.q * I + tid] = sum;
  }
}

template <typename T, int NT, int NC>
__global__ void __launch_bounds__(NT + 32) k_relax(LatView lv, const long long* __restrict__ set_off,
                                              const T* __restrict__ fac, const double2* __restrict__ r,
                                              T* __restrict__ delta, double* __restrict__ P,
                                              T* __restrict__ yglob, long long ystride, const IterCtl* ctl,
                                              int* err, int wait0) {
  relax_body<T, NT, NC>(lv, set_off, fac, r, delta, P, yglob, ystride, ctl, err, blockIdx.x, wait0);
}

// Batched: the sets of every problem of a batch.
template <typename T, int NT, int NC>
__global__ void __launch_bounds__(NT + 32) kb_relax(const BatchProb* __restrict__ Pb, const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = Pb[it.prob];
  const T* fac;
  if constexpr (sizeof(T) == 4) fac = q.f32;
  else fac = q.f64;
  relax_body<T, NT, NC>(q.lv, q.set_off, fac, q.r, (T*)q.delta, q.P, (T*)q.yscratch, y_stride(q.lv), q.ctl,
                        q.err, it.bx, -1);
}

// ---------------------------------------------------------------------------
// The same relaxation on a balanced schedule.  One CTA per set leaves the last
// wave partly idle when the set count is not a multiple of the SM count (256
// sets of 64 x 64 nodes on 152 SMs: two waves, the second on 104 SMs, so the
// SMs are busy 84 % of the kernel's time).  Here one persistent CTA per SM runs
// an equal share of the whole job: the sets' op sequences, laid end to end
// and weighted by their matrix entries, are cut into `grid` equal parts, each
// cut moved to the nearest step boundary after a Linv_j (forward) or Linv_j^T
// (backward) product, where the substitution's state is in global memory
// (y_j in the y scratch, x_j in delta).  A set cut between CTAs g-1 and g has
// its first part (the head) run FIRST by CTA g-1 and its second part (the
// tail) run LAST by CTA g: McNaughton's wrap-around rule, with each CTA
// running head, whole sets, tail.  With every set's cost C at most the share
// T, the head ends at a and the tail starts at T - b >= a (a + b = C), so in a
// balanced run the tail never waits.  The head's CTA releases a per-set flag
// once its part is written; the tail's CTA acquires it (bounded wait) before
// reading the state, and resets it when the set is done.  The CTAs are
// co-resident (cooperative launch) and every head is its CTA's first segment,
// which waits for nothing, so every wait ends.  Each op's arithmetic and the
// P sums are those of relax_body with one copy per matrix, so the results are
// bitwise the same as k_relax's.

__device__ inline int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Bounded wait (about a second) for a set's flag; false if it gave up.
__device__ inline bool set_flag_wait(const int* p) {
  for (int it = 0; it < (1 << 22); ++it) {
    if (ld_acquire_gpu(p) != 0) return true;
    __nanosleep(256);
  }
  return false;
}

template <typename T>
struct SetGeo {
  int I, i0, j0, w, h, nb, nbr, nmat, nops;
  const T* f;   // the factor stored by rows
  const T* ft;  // the copy stored by columns
  T* yg;        // the set's y scratch
};
template <typename T>
__device__ inline SetGeo<T> set_geo(const LatView& lv, const long long* set_off, const T* fac, T* yglob,
                                    long long ystride, int I) {
  SetGeo<T> G;
  G.I = I;
  G.i0 = (I % lv.Mx) * lv.sx;
  G.j0 = (I / lv.Mx) * lv.sy;
  G.w = min(lv.sx, lv.nx - G.i0);
  G.h = min(lv.sy, lv.ny - G.j0);
  G.nb = 2 * G.w;
  G.nbr = y_row(G.nb);
  G.nmat = 2 * G.h - 1;
  G.nops = 2 * G.nmat;
  G.f = fac + set_off[I];
  G.ft = G.f + set_factor_size(G.nb, G.h);
  G.yg = yglob + (size_t)I * ystride;
  return G;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT + 32, 1)
    k_relax_sched(const LatView lv, const long long* __restrict__ set_off, const T* __restrict__ fac,
                  const double2* __restrict__ r, T* __restrict__ delta, double* __restrict__ P,
                  T* __restrict__ yglob, long long ystride, const IterCtl* ctl, int* err,
                  const RelaxSeg* __restrict__ segs, const int* __restrict__ cta_seg, int* flags, int wait0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint64_t bars[NSLOT];
  __shared__ double pred[(VL / 32) * NMODES];
  if (ctl && *(volatile const int*)&ctl->done) return;

  using T2 = typename Vec2<T>::type;
  const int tid = threadIdx.x, lane = tid & 31;
  const bool producer = tid >= NT;
  const int sg0 = cta_seg[blockIdx.x], sg1 = cta_seg[blockIdx.x + 1];
  if (sg0 >= sg1) return;
  // one slot layout for every set: that of the widest
  const RelaxSmem LY = relax_layout<T, 1>(2 * min(lv.sx, lv.nx));
  T* sm = reinterpret_cast<T*>(smraw);
  T* ycur = sm + LY.ycur_off;
  T* zbuf = sm + LY.z_off;
  T* wbuf = sm + LY.w_off;
  T* xbuf = sm + LY.x_off;
  const double* rg = reinterpret_cast<const double*>(r);

  // ---- the producer's cursor over this CTA's ops (thread NT only) ----
  int total = 0, issued = 0, psg = sg0, po = 0;
  bool pfail = false;
  SetGeo<T> PG{};
  auto enter = [&](int sg) {
    // a tail's copies (y rows of the backward pass) read what the head's CTA wrote
    PG = set_geo<T>(lv, set_off, fac, yglob, ystride, segs[sg].I);
    po = segs[sg].o0;
    if (po > 0) {
      if (!set_flag_wait(&flags[PG.I])) pfail = true;
      fence_proxy_async_global();
    }
  };
  auto issue_next = [&]() {
    const int o = po, slot = issued % NSLOT;
    const int k = o < PG.nmat ? o : 2 * PG.nmat - 1 - o;
    const bool fwd = o < PG.nmat;
    const int kind = (k & 1) ? (fwd ? 1 : 3) : (fwd ? 0 : 2);
    uint64_t* bar = &bars[slot];
    const T* src = (fwd ? PG.f : PG.ft) + mat_off(PG.nb, k);
    T* dst = sm + (size_t)slot * LY.slot_elems;
    const int jv = (k + 1) / 2;
    const void* vsrc = fwd ? (const void*)(rg + 2 * ((size_t)(PG.j0 + jv) * lv.nx + PG.i0))
                           : (const void*)(PG.yg + (size_t)(jv - 1) * PG.nbr);
    const uint32_t vbytes = (k & 1) ? (uint32_t)(fwd ? PG.nb * sizeof(double) : PG.nbr * sizeof(T)) : 0u;
    T* vdst = sm + LY.vec_off + (size_t)slot * LY.vec_elems;
    fence_proxy_async_smem();
    if (!fwd && (k & 1)) fence_proxy_async_global();
    const uint32_t bytes = (uint32_t)(kind_size(kind, PG.nb) * sizeof(T));
    mbar_arrive_expect_tx(bar, bytes + vbytes);
    bulk_g2s(dst, src, bytes, bar);
    if (vbytes) bulk_g2s(vdst, vsrc, vbytes, bar);
    ++issued;
    if (++po == segs[psg].o1 && ++psg < sg1) enter(psg);
  };

  if (tid == 0) {
    for (int k = 0; k < NSLOT; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == NT) {
    for (int sg = sg0; sg < sg1; ++sg) total += segs[sg].o1 - segs[sg].o0;
    enter(sg0);
    for (int k = 0; k < NSLOT - 1 && issued < total && !pfail; ++k) issue_next();
  }

  int gop = 0;  // ops of this CTA consumed so far (slot gop % NSLOT)
  bool aborted = false;
  for (int sg = sg0; sg < sg1; ++sg) {
    const RelaxSeg S = segs[sg];
    const SetGeo<T> G = set_geo<T>(lv, set_off, fac, yglob, ystride, S.I);
    // ---- the state the segment starts from ----
    bool bad = tid == NT && pfail;
    if (S.o0 > 0 && tid == 0) bad = !set_flag_wait(&flags[S.I]);
    if (__syncthreads_or(bad)) {
      aborted = true;
      break;
    }
    if (!producer) {
      if (S.o0 == 0) {
        const size_t rowbase0 = 2 * ((size_t)G.j0 * lv.nx + G.i0);  // z = r_0
        for (int t = tid; t < G.nb; t += NT) zbuf[t] = (T)rg[rowbase0 + t];
      } else if (S.o0 <= G.nmat) {
        const T* ys = G.yg + (size_t)((S.o0 - 1) / 2) * G.nbr;  // y_j after Linv_j
        for (int t = tid; t < G.nb; t += NT) ycur[t] = __ldcg(ys + t);
      } else {
        const int j = (2 * G.nmat - S.o0) / 2;  // x_j after Linv_j^T, in delta
        const T* xs = delta + 2 * ((size_t)(G.j0 + j) * lv.nx + G.i0);
        for (int t = tid; t < G.nb; t += NT) xbuf[t] = __ldcg(xs + t);
      }
    }
    __syncthreads();
    const int nb = G.nb, pb = nb / 2;
    for (int o = S.o0; o < S.o1; ++o, ++gop) {
      const uint32_t tries = (gop == 0 && wait0 >= 0) ? (uint32_t)wait0 : MBAR_WAIT_TRIES;
      const bool late = !producer && !mbar_wait_bounded(&bars[gop % NSLOT], (uint32_t)((gop / NSLOT) & 1), tries);
      if (producer) {
        // the slot of op gop - 1 is free since the barrier that ended it
        if (tid == NT && issued < total && !pfail) issue_next();
        if (__syncthreads_or(tid == NT && pfail)) {
          aborted = true;
          break;
        }
        continue;
      }
      const T* M = sm + (size_t)(gop % NSLOT) * LY.slot_elems;
      const T* vstage = sm + LY.vec_off + (size_t)(gop % NSLOT) * LY.vec_elems;
      const int k = o < G.nmat ? o : 2 * G.nmat - 1 - o;
      const bool is_b = (k & 1) != 0;
      const int j = is_b ? (k + 1) / 2 : k / 2;
      constexpr int GR = 4, CH = sizeof(T) == 8 ? 1 : 2;
      if (o < G.nmat) {
        if (is_b) {
          const double* rj = reinterpret_cast<const double*>(vstage);
          rows_times<NT, T, GR, CH, ROW_B>(
              M, ycur, nb, 0, pb, 0, nb, 0, [&](int row) { return (T)rj[row]; },
              [&](int row, T s, T pre) { zbuf[row] = pre - s; });
        } else {
          T* yj = G.yg + (size_t)j * G.nbr;
          rows_times<NT, T, GR, CH, ROW_LINV>(
              M, zbuf, nb, 0, pb, 0, nb, 0, [](int) { return T(0); },
              [&](int row, T s, T) {
                ycur[row] = s;
                yj[row] = s;
              });
        }
      } else {
        if (!is_b) {
          const T* wv = (j == G.h - 1) ? ycur : wbuf;
          T* drow = delta + 2 * ((size_t)(G.j0 + j) * lv.nx + G.i0);
          rows_times<NT, T, GR, CH, ROW_LT>(
              M, wv, nb, 0, pb, 0, nb, 0, [](int) { return T(0); },
              [&](int row, T s, T) {
                xbuf[row] = s;
                drow[row] = s;
              });
        } else {
          const T* yp = vstage;
          rows_times<NT, T, GR, CH, ROW_BT>(
              M, xbuf, nb, 0, pb, 0, nb, 0, [&](int row) { return yp[row]; },
              [&](int row, T s, T pre) { wbuf[row] = pre - s; });
        }
      }
      if (__syncthreads_or(late)) {
        aborted = true;
        break;
      }
    }
    if (aborted) break;
    if (S.o1 < G.nops) {
      // head done: its y rows and delta rows (ordered by the barrier above) go
      // out before the flag
      if (tid == 0) {
        __threadfence();
        st_release_gpu(&flags[S.I], 1);
      }
      continue;
    }
    if (S.o0 > 0 && tid == 0) flags[S.I] = 0;  // both waits on it are past
    if (P == nullptr) continue;
    // P = V^T r (Eq. 7), as in relax_body (delta partly written by another CTA: read from L2)
    __syncthreads();
    const double2 rep = lv.rep[S.I];
    const T2* d2 = reinterpret_cast<const T2*>(delta);
    const int w = G.w, h = G.h, i0 = G.i0, j0 = G.j0;
    for (int vbase = 0; vbase < VL && !producer; vbase += NT) {
      const int v = vbase + tid;
      if (v >= VL) break;
      double pacc[NMODES];
#pragma unroll
      for (int m = 0; m < NMODES; ++m) pacc[m] = 0.0;
      for (int node = v; node < w * h; node += VL) {
        const int jj = node / w, il = node - jj * w;
        const int jn = j0 + jj;
        const size_t nidx = (size_t)jn * lv.nx + i0 + il;
        const double2 rv = r[nidx];
        const T2 dv = __ldcg(d2 + nidx);
        const double xi = fma(lv.L, (double)(i0 + il) + 0.5 * (double)(jn & 1), -rep.x);
        const double eta = fma(lv.L * SQ3_2, (double)jn, -rep.y);
        const double dr = fma((double)dv.x, rv.x, (double)dv.y * rv.y);
        pacc[0] += rv.x;
        pacc[1] += rv.y;
        pacc[2] = fma(xi, rv.x, pacc[2]);
        pacc[3] = fma(eta, rv.x, pacc[3]);
        pacc[4] = fma(xi, rv.y, pacc[4]);
        pacc[5] = fma(eta, rv.y, pacc[5]);
        pacc[6] += dr;
        pacc[7] = fma(xi, dr, pacc[7]);
        pacc[8] = fma(eta, dr, pacc[8]);
      }
#pragma unroll
      for (int m = 0; m < NMODES; ++m) {
        const double sm2 = warp_sum_d(pacc[m]);
        if (lane == 0) pred[(v >> 5) * NMODES + m] = sm2;
      }
    }
    __syncthreads();
    if (tid < NMODES) {
      double sum = 0.0;
      for (int ww = 0; ww < VL / 32; ++ww) sum += pred[ww * NMODES + tid];
      P[(size_t)lv.q * S.I + tid] = sum;
    }
  }
  if (aborted) {
    // the copies still in flight (ops gop .. issued - 1) land before the CTA exits
    if (tid == NT) {
      for (int k = gop; k < issued; ++k) mbar_wait_bounded(&bars[k % NSLOT], (uint32_t)((k / NSLOT) & 1));
      atomicOr(err, (int)DEVERR_TIMEOUT);
    }
  }
}

}  // namespace

size_t relax_smem_bytes(const LatView& lv, bool fp32, int chunks) {
  const int w = region_w_max(lv);
  if (chunks == 2 && !fp32) return relax_layout<double, 2>(2 * w).total_elems * sizeof(double);
  return fp32 ? relax_layout<float>(2 * w).total_elems * sizeof(float)
              : relax_layout<double>(2 * w).total_elems * sizeof(double);
}

// Two copies per matrix apply to the FP64 relaxation when every set width of
// the lattice has a split row r1 (the regular width and the ragged last one).
bool relax_chunks_possible(const LatView& lv, bool fp32) {
  if (fp32 || lv.ov > 0) return false;  // with overlap the region widths vary: one copy
  const int w = lv.sx < lv.nx ? lv.sx : lv.nx;
  const int wr = lv.nx - (lv.Mx - 1) * lv.sx;  // last column of sets
  return chunk_r1<double>(2 * w) > 0 && chunk_r1<double>(2 * wr) > 0;
}

long long relax_y_stride(const LatView& lv) { return y_stride(lv); }

// Cost of op o of a set (nb DOFs per row, nmat matrices per pass): its matrix
// entries (one FMA each) plus a per-op share for the reduction and barrier.
static double op_cost(int nb, int nmat, int o) {
  const int k = o < nmat ? o : 2 * nmat - 1 - o;
  const double e = (k & 1) ? (double)b_row_off(nb, nb) : (double)linv_row_off(nb);
  return e + 8.0 * nb;
}

bool relax_sched_plan(const LatView& lv, int grid, std::vector<RelaxSeg>& segs, std::vector<int>& cta,
                      double* est_sched, double* est_waves) {
  segs.clear();
  cta.clear();
  if (lv.ov != 0 || grid < 2 || lv.M <= grid) return false;
  // per set: the cost at each op boundary
  std::vector<std::vector<double>> pre(lv.M);
  std::vector<double> start(lv.M + 1, 0.0);
  double cmax = 0.0;
  for (int I = 0; I < lv.M; ++I) {
    const int i0 = (I % lv.Mx) * lv.sx, j0 = (I / lv.Mx) * lv.sy;
    const int w = std::min(lv.sx, lv.nx - i0), h = std::min(lv.sy, lv.ny - j0);
    const int nb = 2 * w, nmat = 2 * h - 1, nops = 2 * nmat;
    std::vector<double>& c = pre[I];
    c.assign(nops + 1, 0.0);
    for (int o = 0; o < nops; ++o) c[o + 1] = c[o] + op_cost(nb, nmat, o);
    c[nops] += 12.0 * w * h;  // the P sums
    start[I + 1] = start[I] + c[nops];
    cmax = std::max(cmax, c[nops]);
  }
  const double total = start[lv.M], share = total / grid;
  if (cmax > share) return false;
  // set I: head [0, cut) on CTA hd[I], tail [cut, nops) on CTA hd[I] + 1;
  // cut = nops: the whole set on hd[I]; cut = 0: the whole set on hd[I] + 1
  std::vector<int> hd(lv.M), cut(lv.M);
  for (int I = 0; I < lv.M; ++I) {
    const std::vector<double>& c = pre[I];
    const int nops = (int)c.size() - 1, nmat = nops / 2;
    int g = (int)(start[I] / share);
    g = std::min(g, grid - 1);
    hd[I] = g;
    cut[I] = nops;
    const double x = (g + 1) * share;  // the next CTA's boundary
    if (g + 1 < grid && x < start[I + 1]) {
      // the valid cut (after a Linv_j or a Linv_j^T product) nearest to x
      int best = 0;
      double bd = std::fabs(start[I] - x);
      for (int o = 1; o <= nops; ++o) {
        const bool ok = o == nops || ((o & 1) && o <= nmat) || (!(o & 1) && o > nmat);
        if (!ok) continue;
        const double d = std::fabs(start[I] + c[o] - x);
        if (d < bd) bd = d, best = o;
      }
      cut[I] = best;
    }
  }
  // per CTA: the head it runs first, its whole sets, the tail it runs last
  std::vector<std::vector<RelaxSeg>> head(grid), mid(grid), tail(grid);
  for (int I = 0; I < lv.M; ++I) {
    const int nops = (int)pre[I].size() - 1, g = hd[I];
    if (cut[I] == nops) mid[g].push_back({I, 0, nops, 0});
    else if (cut[I] == 0) mid[g + 1].push_back({I, 0, nops, 0});
    else {
      head[g].push_back({I, 0, cut[I], 0});
      tail[g + 1].push_back({I, cut[I], nops, 0});
    }
  }
  cta.push_back(0);
  double busiest = 0.0;
  for (int g = 0; g < grid; ++g) {
    if (head[g].size() > 1 || tail[g].size() > 1) {
      segs.clear();
      cta.clear();
      return false;
    }
    double cost = 0.0;
    for (auto* v : {&head[g], &mid[g], &tail[g]})
      for (const RelaxSeg& sg : *v) {
        segs.push_back(sg);
        cost += pre[sg.I][sg.o1] - pre[sg.I][sg.o0];
      }
    busiest = std::max(busiest, cost);
    cta.push_back((int)segs.size());
  }
  if (est_sched) *est_sched = busiest / share;
  if (est_waves) {
    // one CTA per set in order, `grid` at a time: the busiest SM's cost
    std::vector<double> load(grid, 0.0);
    for (int I = 0; I < lv.M; ++I) load[I % grid] += start[I + 1] - start[I];
    *est_waves = *std::max_element(load.begin(), load.end()) / share;
  }
  return true;
}

cudaError_t relax_sched_grid(const LatView& lv, bool fp32, int* grid) {
  *grid = 0;
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const size_t smem = relax_smem_bytes(lv, fp32, 1);
  e = fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_relax_sched<float, 256>, 256 + 32, smem)
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_relax_sched<double, 256>, 256 + 32, smem);
  if (e != cudaSuccess) return e;
  *grid = nsm * std::min(per, 1);
  return cudaSuccess;
}

cudaError_t launch_relax_sched(cudaStream_t s, const LatView& lv, const long long* set_off, const double* f64,
                               const float* f32, const double2* r, void* delta, double* P, void* yscratch,
                               const IterCtl* ctl, int* err, const RelaxSeg* segs, const int* cta, int* flags,
                               int grid, int wait0) {
  const bool fp32 = (f32 != nullptr);
  const size_t smem = relax_smem_bytes(lv, fp32, 1);
  const long long ys = relax_y_stride(lv);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(256 + 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  // every CTA resident at once: a tail's CTA may wait for a head's
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (fp32)
    return cudaLaunchKernelEx(&cfg, k_relax_sched<float, 256>, lv, set_off, f32, r, (float*)delta, P,
                              (float*)yscratch, ys, ctl, err, segs, cta, flags, wait0);
  return cudaLaunchKernelEx(&cfg, k_relax_sched<double, 256>, lv, set_off, f64, r, (double*)delta, P,
                            (double*)yscratch, ys, ctl, err, segs, cta, flags, wait0);
}

template <int NC, class F>
static cudaError_t dispatch_nt(int threads, F go) {
  if (threads == 64) go(std::integral_constant<int, 64>(), std::integral_constant<int, NC>());
  else if (threads == 128) go(std::integral_constant<int, 128>(), std::integral_constant<int, NC>());
  else if (threads == 256) go(std::integral_constant<int, 256>(), std::integral_constant<int, NC>());
  else return cudaErrorInvalidValue;
  return cudaSuccess;
}

cudaError_t launch_relax(cudaStream_t s, const LatView& lv, const long long* set_off,
                         const double* f64, const float* f32, const double2* r, void* delta,
                         double* P, void* yscratch, const IterCtl* ctl, int* err, int threads, int chunks,
                         int wait0) {
  const bool fp32 = (f32 != nullptr);
  if (chunks == 2 && !relax_chunks_possible(lv, fp32)) return cudaErrorInvalidValue;
  const size_t smem = relax_smem_bytes(lv, fp32, chunks);
  const long long ys = relax_y_stride(lv);
  auto go = [&](auto nt, auto nc) {
    constexpr int NT = decltype(nt)::value, NC = decltype(nc)::value;
    if (fp32)
      k_relax<float, NT, 1><<<lv.M, NT + 32, smem, s>>>(lv, set_off, f32, r, (float*)delta, P, (float*)yscratch, ys, ctl,
                                                   err, wait0);
    else
      k_relax<double, NT, NC><<<lv.M, NT + 32, smem, s>>>(lv, set_off, f64, r, (double*)delta, P, (double*)yscratch, ys,
                                                     ctl, err, wait0);
  };
  const cudaError_t e = chunks == 2 ? dispatch_nt<2>(threads, go) : dispatch_nt<1>(threads, go);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_batch_relax(cudaStream_t s, bool fp32, int threads, int chunks, size_t smem, const BatchProb* P,
                               const BatchItem* it, int n) {
  if (n <= 0) return cudaSuccess;
  auto go = [&](auto nt, auto nc) {
    constexpr int NT = decltype(nt)::value, NC = decltype(nc)::value;
    if (fp32) kb_relax<float, NT, 1><<<n, NT + 32, smem, s>>>(P, it);
    else kb_relax<double, NT, NC><<<n, NT + 32, smem, s>>>(P, it);
  };
  const cudaError_t e = chunks == 2 ? dispatch_nt<2>(threads, go) : dispatch_nt<1>(threads, go);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t configure_relax(int max_smem) {
  cudaError_t e;
#define HMS_RELAX_ATTR(K)                                                            \
  if ((e = set_max_dynamic_smem(K, max_smem)) != cudaSuccess) return e;
  HMS_RELAX_ATTR((k_relax<float, 64, 1>))
  HMS_RELAX_ATTR((k_relax<float, 128, 1>))
  HMS_RELAX_ATTR((k_relax<float, 256, 1>))
  HMS_RELAX_ATTR((k_relax<double, 64, 1>))
  HMS_RELAX_ATTR((k_relax<double, 128, 1>))
  HMS_RELAX_ATTR((k_relax<double, 256, 1>))
  HMS_RELAX_ATTR((k_relax<double, 64, 2>))
  HMS_RELAX_ATTR((k_relax<double, 128, 2>))
  HMS_RELAX_ATTR((k_relax<double, 256, 2>))
  HMS_RELAX_ATTR((kb_relax<float, 64, 1>))
  HMS_RELAX_ATTR((kb_relax<float, 128, 1>))
  HMS_RELAX_ATTR((kb_relax<float, 256, 1>))
  HMS_RELAX_ATTR((kb_relax<double, 64, 1>))
  HMS_RELAX_ATTR((kb_relax<double, 128, 1>))
  HMS_RELAX_ATTR((kb_relax<double, 256, 1>))
  HMS_RELAX_ATTR((kb_relax<double, 64, 2>))
  HMS_RELAX_ATTR((kb_relax<double, 128, 2>))
  HMS_RELAX_ATTR((kb_relax<double, 256, 2>))
  HMS_RELAX_ATTR((k_relax_sched<float, 256>))
  HMS_RELAX_ATTR((k_relax_sched<double, 256>))
#undef HMS_RELAX_ATTR
  return cudaSuccess;
}

}  // namespace hms
