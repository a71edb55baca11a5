// FP64 symmetric eigensolver (Section 5.2 of the TuckerMPI paper computes all
// eigenpairs of the I_n x I_n Gram matrix; this is a parallel cyclic Jacobi
// method instead of LAPACK's syev) plus the descending sort and the eps rank
// cut of Eq. Un.
//
// Parallel ordering: the round-robin ("circle") tournament.  Storage is kept
// permuted so that the pairs of the current step always sit at positions
// (2j, 2j+1); every step writes the rotated matrix into the other buffer at
// the positions of the next step's pairing, so all pairs of a step are
// disjoint 2x2 blocks and every 2x2 block of A updates independently.
//
// One persistent cooperative kernel runs every sweep with ONE grid barrier
// per step: the thread that produces the off-diagonal entry of a next-step
// pair also recomputes that pair's two new diagonal entries (from their 2x2
// diagonal blocks, with the same expression the diagonal-block thread uses)
// and computes the pair's next rotation.  The eigenvectors are not updated
// every step: each sweep's rotations are logged and replayed once per sweep
// on the rows of V (rows are independent; a warp holds one row in shared
// memory), which takes V off the step's critical path.  Every grid barrier is
// bounded (see GridBarrier).
#include "common.cuh"
#include "kernels.h"

namespace tk {

// Storage position at the next step of the element now at `pos`.  Slots of
// the round robin: position 2k holds slot k, position 2k+1 slot np-1-k; a
// step keeps slot 0 and moves slot s to s+1 (slot np-1 to 1).  In positions:
// 0 stays, an even position moves up by 2 (np-2 goes to np-1), position 1
// goes to 2 and any other odd position moves down by 2.
__device__ __forceinline__ int next_pos(int pos, int np) {
  if (pos & 1) return (pos == 1) ? (np > 2 ? 2 : 1) : pos - 2;
  if (pos == 0) return 0;
  return (pos == np - 2) ? np - 1 : pos + 2;
}

// Rotation (c, s) for the 2x2 block [[app, apq], [apq, aqq]]: the smaller of
// the two angles that annihilate apq (sym.schur2 of Golub & Van Loan,
// Alg. 8.5.1: tau = (aqq - app) / (2 apq), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c).  Skipped (c = 1, s = 0,
// returns false) when |apq| <= max(tol_rel sqrt(|app aqq|), floor_abs).
//
// The angle is computed in FP32 after an exact power-of-two scaling of
// (aqq - app, apq) into range; (c, s) are then made orthonormal to FP64
// rounding by the second-order correction f = 1 - e/2 + 3e^2/8 of
// 1/sqrt(1 + e), e = c^2 + s^2 - 1 (|e| ~ 1e-7, so the neglected term is
// ~1e-21).  The transformation is therefore an exact similarity in FP64; only
// the angle is FP32-accurate, which leaves ~1e-7 |apq| in the annihilated
// entry (kept, and removed by a later sweep).  This keeps the dependent FP64
// chain at ~6 operations (an FP64 operation takes ~64 cycles on this part,
// and the rotation is on the critical path of every step).
// FP64 values seen through their bits: on this part every FP64 instruction,
// a compare or a conversion included, goes through a narrow pipe, so the
// per-step decisions and the FP32 <-> FP64 moves of the rotation use integer
// operations.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
// log2|x| to ~1e-7 (exponent plus the FP32 log2 of the top 23 mantissa bits);
// zero and subnormals come out <= -1023.
__device__ __forceinline__ float log2_abs(double x) {
  const unsigned long long b = abs_bits(x);
  const float m = __int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff));
  return (float)((int)(b >> 52) - 1023) + __log2f(m);
}
// x * 2^sh as FP32 by moving the exponent (mantissa truncated to 23 bits);
// results below the FP32 normal range become 0.
__device__ __forceinline__ float f64_to_f32_shifted(double x, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127 + sh;
  if (e <= 0) return 0.f;
  const unsigned u = (unsigned)(b >> 63) << 31 | (unsigned)(e > 254 ? 254 : e) << 23 |
                     (unsigned)((b >> 29) & 0x7fffff);
  return __uint_as_float(u);
}
// A normal FP32 value as FP64 (exact).
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned long long b = (unsigned long long)(u >> 31) << 63 |
                               (unsigned long long)(((u >> 23) & 0xff) - 127 + 1023) << 52 |
                               (unsigned long long)(u & 0x7fffff) << 29;
  return __longlong_as_double((long long)b);
}

// The rotation test |apq| > max(tol_rel sqrt(|app aqq|), floor_abs): the
// floor exactly (integer compare of magnitudes), the relative part in the
// log2 domain to ~1e-6 (either decision is valid that close to the bound).
__device__ __forceinline__ bool rotation_needed(double app, double aqq, double apq,
                                                float log2_tol_rel, unsigned long long floor_bits) {
  if (!(abs_bits(apq) > floor_bits)) return false;
  return log2_abs(apq) > log2_tol_rel + 0.5f * (log2_abs(app) + log2_abs(aqq));
}

__device__ __forceinline__ bool jacobi_rotation(double app, double aqq, double apq,
                                                float log2_tol_rel, unsigned long long floor_bits,
                                                double& c, double& s) {
  c = 1.0;
  s = 0.0;
  if (!rotation_needed(app, aqq, apq, log2_tol_rel, floor_bits)) return false;
  const double d = aqq - app;
  // scale d and apq by 2^(1023 - E), E the larger biased exponent of the two
  const int ed = (int)(abs_bits(d) >> 52), eb = (int)(abs_bits(apq) >> 52);
  const int sh = 1023 - (ed > eb ? ed : eb);
  const float df = f64_to_f32_shifted(d, sh), bf = f64_to_f32_shifted(apq, sh);
  const float tau = __fdividef(df, 2.f * bf);
  const float atau = fabsf(tau);
  float t = (atau > 1e10f) ? __fdividef(0.5f, atau) : __fdividef(1.f, atau + sqrtf(fmaf(tau, tau, 1.f)));
  t = copysignf(t, tau);
  const float cf = rsqrtf(fmaf(t, t, 1.f));
  const float sf = t * cf;
  if (!(sf != 0.f) || !(cf == cf) || !(bf != 0.f)) return false;   // below FP32 resolution, or NaN
  const double c0 = f32_to_f64(cf), s0 = f32_to_f64(sf);
  const double e = fma(c0, c0, fma(s0, s0, -1.0));
  const double f = fma(e, fma(e, 0.375, -0.5), 1.0);
  c = c0 * f;
  s = s0 * f;
  return true;
}

// Entries of the pair's 2x2 diagonal block [[app, apq], [apq, aqq]] after
// the rotation (c, s): A' = G^T A G with G = [[c, s], [-s, c]].
__device__ __forceinline__ double rot_pp(double app, double apq, double aqq, double c, double s) {
  return fma(c * c, app, fma(-2.0 * c * s, apq, (s * s) * aqq));
}
__device__ __forceinline__ double rot_qq(double app, double apq, double aqq, double c, double s) {
  return fma(s * s, app, fma(2.0 * c * s, apq, (c * c) * aqq));
}
__device__ __forceinline__ double rot_pq(double app, double apq, double aqq, double c, double s) {
  return fma(c * s, app - aqq, (c * c - s * s) * apq);
}

// Block `it` of the upper triangle of 2x2 blocks (column-major order: jb,
// then ja <= jb), the next-step positions of its rows and columns, and the
// entries (bit 2u+v) that become the off-diagonal element of a next-step
// pair.  Depends on positions only, so it is the same at every step.
struct BlockGeom {
  int ja, jb, na0, na1, nb0, nb1;
  unsigned mask;
};
__device__ __forceinline__ BlockGeom block_geom(int64_t it, int np) {
  BlockGeom g;
  int jb = (int)((sqrtf(8.f * (float)it + 1.f) - 1.f) * 0.5f);
  while ((int64_t)(jb + 1) * (jb + 2) / 2 <= it) ++jb;
  while ((int64_t)jb * (jb + 1) / 2 > it) --jb;
  g.jb = jb;
  g.ja = (int)(it - (int64_t)jb * (jb + 1) / 2);
  const int na[2] = {next_pos(2 * g.ja, np), next_pos(2 * g.ja + 1, np)};
  const int nb[2] = {next_pos(2 * jb, np), next_pos(2 * jb + 1, np)};
  g.na0 = na[0]; g.na1 = na[1]; g.nb0 = nb[0]; g.nb1 = nb[1];
  unsigned mask = 0;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      if (g.ja == jb && !(u == 0 && v == 1)) continue;
      const int r = na[u], c = nb[v];
      if ((r >> 1) == (c >> 1) && r != c) mask |= 1u << (2 * u + v);
    }
  g.mask = mask;
  return g;
}

struct JacobiArgs {
  double* A[2];       // np x np row-major, ping-pong
  double* V;          // n x np row-major (rows: coordinates, cols: storage positions)
  double* rot[2];     // 2 * P: c, s of the current / next step
  double* log;        // (np - 1) * P * 2: c, s of every step of the current sweep
  unsigned* counts;   // non-skipped rotations per sweep (max_sweeps + 1 entries, zeroed)
  int* info;          // [0] sweeps, [1] converged, [2] final A buffer, [3] dummy position
  const double* fro2; // ||S||_F^2
  GridBarrier bar;
  unsigned long long poll_limit;   // polls before a grid barrier gives up
  int n, np, max_sweeps, vwarps;
  double tol_rel, tol_abs;
};

__device__ __forceinline__ void count_rotation(unsigned* counts, int idx, int max_sweeps) {
  if (idx <= max_sweeps) atomicAdd(&counts[idx], 1u);
}

constexpr int VGROUP = 8;   // log entries a lane loads at once in the V pass
constexpr int VROWS = 2;    // target V rows per CTA

__global__ void __launch_bounds__(256, 1) k_jacobi(JacobiArgs a) {
  extern __shared__ __align__(16) double vsm[];
  const int n = a.n, np = a.np, P = np >> 1;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
  const double floor_abs = a.tol_abs * sqrt(*a.fro2);
  const unsigned long long floor_bits = abs_bits(floor_abs);
  const float log2_tol = (a.tol_rel > 0.0) ? log2f((float)a.tol_rel) : -INFINITY;
  const int64_t nblk = (int64_t)P * (P + 1) / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* const A0 = a.A[0];
  double* const A1 = a.A[1];
  double* const rot0 = a.rot[0];
  double* const rot1 = a.rot[1];
  unsigned gen = 0;
  int cur = 0, rc = 0;
  int dpos = (n & 1) ? n : -1;   // dummy index (odd n) sits at position n initially
  int sweeps = 0, converged = 0;
  const BlockGeom g0 = block_geom(gtid < nblk ? gtid : 0, np);   // this thread's first block

  // prologue: rotations of step 0
  for (int64_t j = gtid; j < P; j += gsz) {
    const int p = 2 * (int)j;
    const double* A = A0;
    double c, s;
    if (jacobi_rotation(A[(int64_t)p * np + p], A[(int64_t)(p + 1) * np + p + 1],
                        A[(int64_t)p * np + p + 1], log2_tol, floor_bits, c, s))
      count_rotation(a.counts, 0, a.max_sweeps);
    reinterpret_cast<double2*>(rot0)[j] = make_double2(c, s);
  }
  if (!grid_sync(a.bar, gen, a.poll_limit)) return;

  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    // the sweep's step-0 rotations into the log
    for (int64_t j = gtid; j < P; j += gsz) {
      const double* Rc = rc ? rot1 : rot0;
      reinterpret_cast<double2*>(a.log)[j] = reinterpret_cast<const double2*>(Rc)[j];
    }
    for (int t = 0; t < np - 1; ++t) {
      // pointer selects, not runtime-indexed parameter arrays (those would go
      // through local memory, which the barrier's acquire sends back to L2)
      const double* A = cur ? A1 : A0;
      double* An = cur ? A0 : A1;
      const double* R = rc ? rot1 : rot0;
      double* Rn = rc ? rot0 : rot1;
      const bool last = (t == np - 2);
      const int next_sweep = last ? sweep + 1 : sweep;
      for (int64_t it = gtid; it < nblk; it += gsz) {
        const BlockGeom g = (it == gtid) ? g0 : block_geom(it, np);
        const int ja = g.ja, jb = g.jb, pa = 2 * ja, pb = 2 * jb;
        const int na[2] = {g.na0, g.na1};
        const int nb[2] = {g.nb0, g.nb1};
        unsigned mask = g.mask;
        // every load of the step is issued here, in one round trip: the block,
        // and for a block that feeds a next rotation the diagonal blocks of
        // pairs ja and jb (their new diagonal entries)
        const double2 r0 = *reinterpret_cast<const double2*>(A + (int64_t)pa * np + pb);
        const double2 r1 = *reinterpret_cast<const double2*>(A + (int64_t)(pa + 1) * np + pb);
        double2 da = make_double2(0.0, 0.0), db = make_double2(0.0, 0.0);
        double daq = 0.0, dbq = 0.0;
        if (mask && ja != jb) {
          da = *reinterpret_cast<const double2*>(A + (int64_t)pa * np + pa);        // app, apq
          daq = A[(int64_t)(pa + 1) * np + pa + 1];                                 // aqq
          db = *reinterpret_cast<const double2*>(A + (int64_t)pb * np + pb);
          dbq = A[(int64_t)(pb + 1) * np + pb + 1];
        }
        const double a00 = r0.x, a01 = r0.y, a10 = r1.x, a11 = r1.y;
        double nv[2][2];
        const double2 Ra = reinterpret_cast<const double2*>(R)[ja];
        const double2 Rb = reinterpret_cast<const double2*>(R)[jb];
        // a skipped rotation is exactly (c, s) = (1, 0), which the update
        // formulas reproduce exactly; a warp whose blocks all have skipped
        // rotations (most warps of the later sweeps) copies and issues no
        // FP64 instruction.  The test is an integer compare of s's bits.
        const bool rot_a = __double_as_longlong(Ra.y) != 0, rot_b = __double_as_longlong(Rb.y) != 0;
        const bool any_rot = __any_sync(__activemask(), rot_a || rot_b);
        if (ja == jb) {
          const double c = Ra.x, s = Ra.y;
          double d0 = a00, d1 = a11, off = a01;
          if (any_rot) {
            d0 = rot_pp(a00, a01, a11, c, s);
            d1 = rot_qq(a00, a01, a11, c, s);
            off = rot_pq(a00, a01, a11, c, s);
          }
          nv[0][0] = d0; nv[1][1] = d1; nv[0][1] = off; nv[1][0] = off;
          An[(int64_t)na[0] * np + na[0]] = d0;
          An[(int64_t)na[1] * np + na[1]] = d1;
          An[(int64_t)na[0] * np + na[1]] = off;
          An[(int64_t)na[1] * np + na[0]] = off;
        } else {
          const double ca = Ra.x, sa = Ra.y;
          const double cb = Rb.x, sb = Rb.y;
          if (any_rot) {
            const double q00 = ca * a00 - sa * a10, q01 = ca * a01 - sa * a11;
            const double q10 = sa * a00 + ca * a10, q11 = sa * a01 + ca * a11;
            nv[0][0] = q00 * cb - q01 * sb; nv[0][1] = q00 * sb + q01 * cb;
            nv[1][0] = q10 * cb - q11 * sb; nv[1][1] = q10 * sb + q11 * cb;
          } else {
            nv[0][0] = a00; nv[0][1] = a01; nv[1][0] = a10; nv[1][1] = a11;
          }
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              An[(int64_t)na[u] * np + nb[v]] = nv[u][v];
              An[(int64_t)nb[v] * np + na[u]] = nv[u][v];
            }
        }
        // next-step pairs whose off-diagonal entry this block produced: only
        // these threads run the rotation (a data-dependent loop, so the FP64
        // chain is not executed predicated by every thread)
        while (mask) {
          const int k = __ffs(mask) - 1;
          mask &= mask - 1;
          const int u = k >> 1, v = k & 1;
          const int r = na[u];
          const int jn = r >> 1;
          double dr, dc;
          if (ja == jb) {
            dr = nv[0][0];
            dc = nv[1][1];
          } else {
            dr = !rot_a ? (u ? daq : da.x)
                        : (u ? rot_qq(da.x, da.y, daq, Ra.x, Ra.y) : rot_pp(da.x, da.y, daq, Ra.x, Ra.y));
            dc = !rot_b ? (v ? dbq : db.x)
                        : (v ? rot_qq(db.x, db.y, dbq, Rb.x, Rb.y) : rot_pp(db.x, db.y, dbq, Rb.x, Rb.y));
          }
          const double off = (k == 0) ? nv[0][0] : (k == 1) ? nv[0][1] : (k == 2) ? nv[1][0] : nv[1][1];
          const bool r_first = (r & 1) == 0;
          double cn, sn;
          if (jacobi_rotation(r_first ? dr : dc, r_first ? dc : dr, off, log2_tol, floor_bits, cn,
                              sn))
            count_rotation(a.counts, next_sweep, a.max_sweeps);
          reinterpret_cast<double2*>(Rn)[jn] = make_double2(cn, sn);
          if (!last) {
            a.log[((int64_t)(t + 1) * P + jn) * 2] = cn;
            a.log[((int64_t)(t + 1) * P + jn) * 2 + 1] = sn;
          }
        }
      }
      if (dpos >= 0) dpos = next_pos(dpos, np);
      cur ^= 1;
      rc ^= 1;
      if (!grid_sync(a.bar, gen, a.poll_limit)) return;
    }
    sweeps = sweep + 1;
    // replay the sweep's rotations on the rows of V (V' = V J_0 ... J_{np-2})
    if (warp < a.vwarps) {
      double* b0 = vsm + (size_t)warp * 2 * np;
      double* b1 = b0 + np;
      // rows spread over all CTAs first (the pass is FP64-throughput bound:
      // a row per warp on as many SMs as possible)
      for (int row = blockIdx.x + gridDim.x * warp; row < n; row += gridDim.x * a.vwarps) {
        double* vr = a.V + (int64_t)row * np;
        for (int cidx = lane; cidx < np; cidx += 32) b0[cidx] = vr[cidx];
        __syncwarp();
        // flattened (step, group) loop; the next group's (c, s) loads are in
        // flight while the current group is applied
        const int G = (P + 32 * VGROUP - 1) / (32 * VGROUP);
        const int64_t total = (int64_t)(np - 1) * G;
        const double2* lg = reinterpret_cast<const double2*>(a.log);
        double2 cs[VGROUP], csn[VGROUP];
#pragma unroll
        for (int k = 0; k < VGROUP; ++k) {
          const int j = 32 * k + lane;
          cs[k] = (j < P) ? lg[j] : make_double2(1.0, 0.0);
        }
        int t1 = 0, g1 = 0;   // (step, group) of the prefetch
        for (int64_t it = 0; it < total; ++it) {
          const int j0 = g1 * 32 * VGROUP;
          if (++g1 == G) { g1 = 0; ++t1; }
          if (it + 1 < total) {
            const int j1 = g1 * 32 * VGROUP;
#pragma unroll
            for (int k = 0; k < VGROUP; ++k) {
              const int j = j1 + 32 * k + lane;
              csn[k] = (j < P) ? lg[(int64_t)t1 * P + j] : make_double2(1.0, 0.0);
            }
          }
#pragma unroll
          for (int k = 0; k < VGROUP; ++k) {
            const int j = j0 + 32 * k + lane;
            // identity rotations (most of the later sweeps) are copies; the
            // FP64 arithmetic is issued only if a lane of the group rotates
            const bool rot = __any_sync(0xffffffffu, __double_as_longlong(cs[k].y) != 0);
            if (j < P) {
              const double2 v = reinterpret_cast<const double2*>(b0)[j];
              double n0 = v.x, n1 = v.y;
              if (rot) {
                n0 = cs[k].x * v.x - cs[k].y * v.y;
                n1 = cs[k].y * v.x + cs[k].x * v.y;
              }
              b1[next_pos(2 * j, np)] = n0;
              b1[next_pos(2 * j + 1, np)] = n1;
            }
          }
#pragma unroll
          for (int k = 0; k < VGROUP; ++k) cs[k] = csn[k];
          if (j0 + 32 * VGROUP >= P) {   // last group of step t
            __syncwarp();
            double* tmp = b0; b0 = b1; b1 = tmp;
          }
        }
        for (int cidx = lane; cidx < np; cidx += 32) vr[cidx] = b0[cidx];
        __syncwarp();
      }
    }
    if (!grid_sync(a.bar, gen, a.poll_limit)) return;
    if (ld_acquire_u32(&a.counts[sweep]) == 0u) { converged = 1; break; }
  }
  if (gtid == 0) {
    a.info[0] = sweeps;
    a.info[1] = converged;
    a.info[2] = cur;
    a.info[3] = dpos;
  }
}

// Padded copy S (n x n) -> A (np x np) and V = [I | 0] (n x np).
__global__ void k_jacobi_init(const double* __restrict__ S, int n, int np, double* __restrict__ A,
                              double* __restrict__ V) {
  int64_t tot = (int64_t)np * np;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / np, j = e % np;
    A[e] = (i < n && j < n) ? S[i * n + j] : 0.0;
    if (i < n) V[i * np + j] = (i == j) ? 1.0 : 0.0;
  }
}

// Ranks eigenvalues (descending; ties by position) and writes them out.
__global__ void __launch_bounds__(1024) k_eig_rank(const double* __restrict__ A, int n, int np,
                                                   const int* __restrict__ info,
                                                   int* __restrict__ rank, double* __restrict__ w) {
  const int dpos = info[3];
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    if (p == dpos) { rank[p] = -1; continue; }
    const double lp = A[(int64_t)p * np + p];
    int r = 0;
    for (int q = 0; q < np; ++q) {
      if (q == dpos || q == p) continue;
      const double lq = A[(int64_t)q * np + q];
      r += (lq > lp) || (lq == lp && q < p);
    }
    rank[p] = r;
    w[r] = lp;
  }
}

// V_out (n x n column-major) column rank[p] = V column p.
__global__ void k_eig_gather(const double* __restrict__ V, int n, int np, const int* __restrict__ rank,
                             double* __restrict__ Vout) {
  int64_t tot = (int64_t)n * np;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / np;
    int p = (int)(e % np);
    int r = rank[p];
    if (r >= 0) Vout[i + (int64_t)n * r] = V[e];
  }
}

// Eq. Un: R = min{R in 1..n : sum_{i>=R} w_i <= thr}; the tail is
// accumulated from the smallest eigenvalue up.  out_R[0] = R, out_d[0] = tail(R).
// With fixed_R > 0 the rank is given (rank-specified variant) and only the
// discarded tail is computed.
__global__ void k_rank_cut(const double* __restrict__ w, int n, double thr, int fixed_R,
                           int64_t* out_R, double* out_d, double* tail) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  tail[n] = 0.0;
  for (int i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + w[i];
  int R = n;
  if (fixed_R > 0) {
    R = fixed_R;
  } else {
    for (int r = 1; r <= n; ++r)
      if (tail[r] <= thr) { R = r; break; }
  }
  out_R[0] = R;
  out_d[0] = tail[R];
}

namespace {
struct JacobiLayout {
  double *A0, *A1, *V, *rot0, *rot1, *log;
  int* rank;
};
JacobiLayout jacobi_layout(int n, double* work) {
  const size_t np = n + (n & 1), P = np / 2;
  JacobiLayout L;
  L.A0 = work;
  L.A1 = L.A0 + np * np;
  L.V = L.A1 + np * np;
  L.rot0 = L.V + (size_t)n * np;
  L.rot1 = L.rot0 + 2 * P;
  L.log = L.rot1 + 2 * P;
  L.rank = (int*)(L.log + 2 * P * (np > 1 ? np - 1 : 1));
  return L;
}
int vpass_warps(int np) {
  const size_t per_warp = 2 * (size_t)np * sizeof(double);
  size_t w = (96 * 1024) / per_warp;
  if (w > 8) w = 8;
  if (w < 1) w = 1;
  return (int)w;
}
}  // namespace

size_t jacobi_work_bytes(int n) {
  const size_t np = n + (n & 1), P = np / 2;
  return sizeof(double) * (2 * np * np + (size_t)n * np + 4 * P + 2 * P * (np > 1 ? np - 1 : 1)) +
         sizeof(int) * (np + 4);
}

int jacobi_max_n() { return 8192; }

cudaError_t launch_jacobi(const double* S, int n, double* work, const double* fro2, unsigned* words,
                          int max_sweeps, double tol_rel, double tol_abs, int num_sms,
                          double* w_out, double* V_out, int* info_dev, cudaStream_t st,
                          unsigned long long poll_limit) {
  const int np = n + (n & 1);
  const JacobiLayout L = jacobi_layout(n, work);
  // words: [0] barrier count, [1] barrier gen, [2] err, [3..] per-sweep counts
  cudaError_t e = cudaMemsetAsync(words, 0, sizeof(unsigned) * (3 + max_sweeps + 2), st);
  if (e != cudaSuccess) return e;
  k_jacobi_init<<<256, 256, 0, st>>>(S, n, np, L.A0, L.V);
  count_launches(max_sweeps > 0 ? 2 : 1);
  JacobiArgs a;
  a.A[0] = L.A0; a.A[1] = L.A1; a.V = L.V;
  a.rot[0] = L.rot0; a.rot[1] = L.rot1;
  a.log = L.log;
  a.counts = words + 3;
  a.info = info_dev;
  a.fro2 = fro2;
  a.bar = GridBarrier{words, words + 1, words + 2};
  a.poll_limit = poll_limit;
  a.n = n; a.np = np; a.max_sweeps = max_sweeps;
  a.tol_rel = tol_rel; a.tol_abs = tol_abs;
  a.vwarps = vpass_warps(np);
  const size_t smem = (size_t)a.vwarps * 2 * np * sizeof(double);
  e = allow_max_dyn_smem((const void*)k_jacobi);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  const int64_t P = np / 2;
  const int64_t items = P * (P + 1) / 2;
  int64_t want = (items + 255) / 256;
  // the V pass is FP64-throughput bound: at most VROWS rows per CTA where
  // the SM count allows
  if (want < (n + VROWS - 1) / VROWS) want = (n + VROWS - 1) / VROWS;
  const int64_t cap = num_sms;   // one CTA per SM: fewer arrivals per barrier
  const int grid = (int)(want < 1 ? 1 : (want > cap ? cap : want));
  if (max_sweeps > 0) {
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((void*)k_jacobi, dim3(grid), dim3(256), args, smem, st);
    if (e != cudaSuccess) return e;
  } else {
    int h[4] = {0, 0, 0, (n & 1) ? n : -1};
    e = cudaMemcpyAsync(info_dev, h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_eig_finish(int n, double* work, const int* info_host, int* info_dev,
                              double* w_out, double* V_out, cudaStream_t st) {
  const int np = n + (n & 1);
  const JacobiLayout L = jacobi_layout(n, work);
  const double* A = info_host[2] ? L.A1 : L.A0;
  k_eig_rank<<<1, 1024, 0, st>>>(A, n, np, info_dev, L.rank, w_out);
  count_launches(2);
  int64_t tot = (int64_t)n * np;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_eig_gather<<<blocks, 256, 0, st>>>(L.V, n, np, L.rank, V_out);
  return cudaGetLastError();
}

cudaError_t launch_rank_cut(const double* w, int n, double thr, int fixed_R, int64_t* out_R,
                            double* out_d, double* tail, cudaStream_t st) {
  k_rank_cut<<<1, 32, 0, st>>>(w, n, thr, fixed_R, out_R, out_d, tail);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tk
