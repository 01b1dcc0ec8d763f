// Register-resident sweep steps for small bonds (one warp, no block barriers).
//
// For small chi the matrices of a sweep step fit one warp with one element
// per lane, so a whole factorisation runs in registers with warp-shuffle
// reductions instead of shared-memory passes separated by block barriers.
// On this part an FP64 warp instruction holds the FP64 pipe for many cycles
// whatever the number of active lanes, so the layouts below keep every lane
// busy and the reductions pair their operands (two or four sums for the
// price of one butterfly):
//  * tiny_qr_factor / tiny_q_store: rank-revealing Householder QR of an
//                   m x n matrix, m <= 8, n <= 4; column c on lanes 8c..8c+7,
//                   row i = lane & 7.  With two or more warps the thin Q is
//                   formed and stored by warp 1 one step behind, off the
//                   sweep's critical path (R feeds the next step, Q does not).
//  * tiny_svd_step: one SVD-sweep step, one-sided Jacobi on the rows of an
//                   r x c matrix with the r x r rotation accumulator beside
//                   it (r <= 4, c + r <= 8); row p on lanes 8p..8p+7, lane
//                   8p+j holds Mat[p][j] (j < c) or U[p][j-c].
// The arithmetic rules (reflector and its phase floor, pivoting and rank
// stop, rotation angle and normalisation, pair order, convergence and noise
// floor, rank rule, truncation bookkeeping) are those of the block-cooperative
// routines in gmps_kernels.cu; only the data placement and the reduction order
// differ.  Included by gmps_kernels.cu inside namespace gmps, after its
// helpers.
#pragma once


template <class T>
__device__ __forceinline__ cx<T> shcx(cx<T> v, int src) {
  return mk<T>(shidx(v.re, src), shidx(v.im, src));
}
template <class T>
__device__ __forceinline__ cx<T> shcx_x(cx<T> v, int o) {
  return mk<T>(shx(v.re, o), shx(v.im, o));
}
// sum over each aligned group of 8 lanes (all 8 lanes get it)
template <class T>
__device__ __forceinline__ T sum8(T v) {
  v += shx(v, 4);
  v += shx(v, 2);
  v += shx(v, 1);
  return v;
}
// Sums of two values over each aligned group of 8 lanes in three adds: lanes
// 0..3 of the group end with the sum of v0, lanes 4..7 with the sum of v1.
template <class T>
__device__ __forceinline__ T sum8x2(T v0, T v1, int j) {
  const bool hi = (j & 4) != 0;
  T t = (hi ? v1 : v0) + shx(hi ? v0 : v1, 4);
  t += shx(t, 2);
  t += shx(t, 1);
  return t;
}
// Sums of four values over each aligned group of 8 lanes in four adds: lanes
// 0,1 end with the sum of v0, 2,3 of v1, 4,5 of v2, 6,7 of v3.
template <class T>
__device__ __forceinline__ T sum8x4(T v0, T v1, T v2, T v3, int j) {
  const bool h4 = (j & 4) != 0;
  const T a0 = (h4 ? v2 : v0) + shx(h4 ? v0 : v2, 4);
  const T a1 = (h4 ? v3 : v1) + shx(h4 ? v1 : v3, 4);
  const bool h2 = (j & 2) != 0;
  T t = (h2 ? a1 : a0) + shx(h2 ? a0 : a1, 2);
  t += shx(t, 1);
  return t;
}
template <class T>
__device__ __forceinline__ T pick4(T a0, T a1, T a2, T a3, int i) {
  return i == 0 ? a0 : (i == 1 ? a1 : (i == 2 ? a2 : a3));
}
// |x0|^2 > phase_floor |x|^2 for the Householder phase (both non-negative);
// for doubles with |x|^2 above 2^-900 the floor 2^-120 is an exponent shift
template <class T>
__device__ __forceinline__ bool above_phase_floor(T a2, T s) {
  return a2 > K<T>::phase_floor() * s;
}
template <>
__device__ __forceinline__ bool above_phase_floor<double>(double a2, double s) {
  const long long sb = __double_as_longlong(s);
  if (sb > (124LL << 52)) return __double_as_longlong(a2) > sb - (120LL << 52);
  return a2 > K<double>::phase_floor() * s;
}

// Rank-revealing QR of W (m x n), m <= 8, n <= 4, by warp 0; lane 8c + i
// brings W[i][c] in w0 (zero outside the matrix).  Same rules as
// qr_rank_revealing: the pivot is the column of largest remaining norm
// (compared exactly here, through FP32 images there), the factorisation stops
// at the first step whose largest remaining squared norm is <= floor_rel2
// times the largest input column's.  Each reflector is stored scaled by
// sqrt(tau) (H = I - v v^dag).  Writes R P^T (p x n, leading dim n) to Rp and
// leaves the reflectors in the lanes' `a` (column jj's lanes, rows >= jj) for
// tiny_q_store; returns p (the same in every lane).
template <class T>
__device__ int tiny_qr_factor(cx<T> w0, int m, int n, T floor_rel2, cx<T>* Rp, cx<T>& a_out) {
  const int lane = threadIdx.x & 31;
  const int c = lane >> 3, i = lane & 7;
  const bool live = c < n && i < m;
  const cx<T> zero = mk<T>(0, 0);
  cx<T> a = w0;
  int pc = c;  // original index of the column now at position c
  cx<T> be0 = zero, be1 = zero, be2 = zero, be3 = zero;
  const int pmax = min(m, n);
  int rank = pmax;
  T flr = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j >= pmax) break;
    // squared norms of every column over rows >= j, seen by all lanes
    const T s = sum8((live && i >= j) ? abs2(a) : (T)0);
    const T cn0 = shidx(s, 0), cn1 = shidx(s, 8), cn2 = shidx(s, 16), cn3 = shidx(s, 24);
    int best = j;
    T sb = pick4(cn0, cn1, cn2, cn3, j);
#pragma unroll
    for (int cc = 1; cc < 4; ++cc) {
      const T v = pick4(cn0, cn1, cn2, cn3, cc);
      if (cc > j && cc < n && nn_gt(v, sb)) {
        sb = v;
        best = cc;
      }
    }
    if (j == 0) {
      flr = sb * floor_rel2;
    } else if (!nn_gt(sb, flr)) {
      rank = j;
      break;
    }
    if (best != j) {  // swap columns j and best (warp-uniform)
      const cx<T> fb = shcx(a, best * 8 + i), fj = shcx(a, j * 8 + i);
      const int pb = __shfl_sync(0xffffffffu, pc, best * 8), pj = __shfl_sync(0xffffffffu, pc, j * 8);
      if (c == j) {
        a = fb;
        pc = pb;
      } else if (c == best) {
        a = fj;
        pc = pj;
      }
    }
    const bool colj = c == j && i >= j && i < m;
    // reflector from the pivot column (scaled by a power of two first when the
    // arithmetic has FP32's exponent range)
    T sx = sb;
    int em = 0;
    bool scl = false;
    if (K<T>::kScaleColumns) {
      int e = -2000;
      if (colj) {
        if (a.re != (T)0) e = expo_abs(a.re);
        if (a.im != (T)0) e = max(e, expo_abs(a.im));
      }
      e = __reduce_max_sync(0xffffffffu, e);
      if (e > -2000) {
        scl = true;
        em = e;
        if (colj) a = cscale(a, pow2<T>(-em));
        sx = shidx(sum8(colj ? abs2(a) : (T)0), j * 8);
      }
    }
    const cx<T> x0 = shcx(a, j * 8 + j);
    const T a2 = abs2(x0);
    cx<T> b = zero;
    if (nn_gt(sx, K<T>::tiny2())) {
      // 1/|x| and 1/|x_j| in one instruction stream (lanes 0..15 and 16..31)
      const bool usep = above_phase_floor(a2, sx);
      const T r = rsqrt((lane < 16 || !usep) ? sx : a2);
      const T inv = shidx(r, 0), ia = shidx(r, 16);
      const T nrm = sx * inv;
      cx<T> ph = mk<T>(1, 0);
      T ax0 = 0;
      if (usep) {
        ax0 = a2 * ia;
        ph = cscale(x0, ia);
      }
      b = cscale(ph, -nrm);
      // v = x - beta e_j scaled by sqrt(tau), tau = 1/(|x| (|x| + |x_j|))
      const T w = rsqrt(nrm * (nrm + ax0));
      if (colj) a = cscale(i == j ? csub(x0, b) : a, w);
    }
    if (scl) b = cscale(b, pow2<T>(em));
    if (j == 0) be0 = b;
    if (j == 1) be1 = b;
    if (j == 2) be2 = b;
    if (j == 3) be3 = b;
    // columns right of j: x <- x - v (v^dag x)
    const cx<T> vi = shcx(a, j * 8 + i);
    const bool upd = live && c > j && i >= j;
    const cx<T> pr = upd ? cmacc(zero, vi, a) : zero;
    const T t = sum8x2(pr.re, pr.im, i);
    const int g0 = lane & ~7;
    const cx<T> d = mk<T>(shidx(t, g0), shidx(t, g0 + 4));
    if (upd) a = cmac(a, vi, mk<T>(-d.re, -d.im));
  }
  const int p = rank;
  // R P^T: row i < p; the column at position c is original column pc
  if (live && i < p) Rp[i * n + pc] = c > i ? a : (c == i ? pick4(be0, be1, be2, be3, i) : zero);
  a_out = a;
  return p;
}

// The thin Q (m x p, row-major, to dst) from the reflectors that
// tiny_qr_factor left in the lanes' `a`; any one warp can run it.  Column c =
// H_0 ... H_{p-1} e_c is built in the lanes of column c; the
  // first factor applied is H_{p-1} e_c = e_c - v conj(v_c) (no reduction).
template <class T, class S>
__device__ void tiny_q_store(cx<T> a, int m, int p, S* dst, unsigned long long key) {
  const int lane = threadIdx.x & 31;
  const int c = lane >> 3, i = lane & 7;
  const cx<T> zero = mk<T>(0, 0);
  cx<T> q;
  {
    const cx<T> vl = shcx(a, (p - 1) * 8 + i), vc = shcx(a, (p - 1) * 8 + c);
    const bool in = i >= p - 1 && i < m && c >= p - 1;
    q = mk<T>((c == i) ? (T)1 : (T)0, 0);
    if (in) q = cmac(q, vl, mk<T>(-vc.re, vc.im));  // - v_i conj(v_c)
  }
#pragma unroll
  for (int jj = 2; jj >= 0; --jj) {
    if (jj >= p - 1) continue;
    const cx<T> vj = shcx(a, jj * 8 + i);
    const bool in = i >= jj && i < m;
    const cx<T> pr = in ? cmacc(zero, vj, q) : zero;
    const T t = sum8x2(pr.re, pr.im, i);
    const int g0 = lane & ~7;
    const cx<T> d = mk<T>(shidx(t, g0), shidx(t, g0 + 4));
    if (in) q = cmac(q, vj, mk<T>(-d.re, -d.im));
  }
  if (c < p && i < m) st_site(dst + i * p + c, q, key, i * p + c);
}

// Hand-off of a small QR step between warps: two buffers (by site parity),
// each the 32 lanes' reflector registers followed by (p, m).
template <class T>
__device__ __forceinline__ cx<T>* tbuf_regs(unsigned char* tb, int b) {
  return (cx<T>*)(tb + b * (32 * sizeof(cx<T>) + 16));
}
template <class T>
__device__ __forceinline__ int* tbuf_meta(unsigned char* tb, int b) {
  return (int*)(tb + b * (32 * sizeof(cx<T>) + 16) + 32 * sizeof(cx<T>));
}

// One step of the SVD sweep at site l (rl <= 4, c = 2 kr, c + rl <= 8), by
// warp 0: Mat = A_l (rl x 2 x rr) * US (rr x kr), one-sided Jacobi on its
// rows with U accumulated beside it, the rank rule, and the outputs: site l
// = rows of V^dag (k x c), US = U^dag[:, perm] sigma (rl x k), chi[l] = k and
// misc[4] = k.  Same rules as the block path of sweep_pair.
template <class T, class S, class CR>
__device__ void tiny_svd_step(Blk<T, S>& B, int l, int rl, int rr, int kr) {
  const InstDesc& d = *B.d;
  const int c = 2 * kr;
  const int lane = threadIdx.x & 31, p = lane >> 3, j = lane & 7;
  const bool row = p < rl;
  const bool inM = row && j < c;
  const bool inU = row && j >= c && j < c + rl;
  const cx<T> zero = mk<T>(0, 0);
  S* A = B.slot(l);
  cx<T> x = zero;
  if (inM) {
    const int s = j >= kr ? 1 : 0, jj = j - s * kr;
    cx<CR> acc = mk<CR>(0, 0);
    for (int a = 0; a < rr; ++a) acc = cmac(acc, ld<CR>(A + (p * 2 + s) * rr + a), cvt<CR>(B.US[a * kr + jj]));
    x = cvt<T>(acc);
  } else if (inU) {
    x = mk<T>((j - c == p) ? (T)1 : (T)0, 0);
  }
  // noise floor for skipping rotations: (max(m,n) eps / 4)^2 times the
  // squared Frobenius norm of the swept matrices, measured at the first site
  T frob;
  if (l == B.n - 1) {
    frob = gsum(inM ? abs2(x) : (T)0, 32);
    if (lane == 0) B.tmisc[9] = frob;
  } else {
    frob = B.tmisc[9];
  }
  const T fl = rank_floor(B, rl, c) * (T)0.25f;
  const T skip2 = frob * fl * fl;
  // Jacobi sweeps; the round-robin rounds pair row p with p ^ dx.  own2 keeps
  // this row's |x_p|^2 from the latest round (sigma_p^2 once a sweep ends
  // without rotating)
  int sw = 0;
  T own2 = 0;
  // a single pair (rl == 2) whose rotation had |g| <= 2^-32 sqrt(a b) is
  // done: the FP32 angle leaves at most ~1.6 * 2^-22 of that off-diagonal and
  // FP64 rounding ~2^-53, both far below the rotation threshold, so the sweep
  // that would confirm it rotates nothing and is skipped (the row norms are
  // then summed afresh, as that sweep's Gram diagonal would give them)
  bool done_early = false;
  if (rl >= 2) {
    sw = -1;
    const int nround = rl == 2 ? 1 : 3;
    for (int sweep = 0; sweep < d.max_sweeps; ++sweep) {
      bool rotated = false;
      for (int t = 0; t < nround; ++t) {
        const int dx = nround == 1 ? 1 : 3 - t;
        const int q = p ^ dx;
        const bool isP = p < q;
        const int lp = 8 * (isP ? p : q), lq = 8 * (isP ? q : p);
        const cx<T> y = shcx_x(x, 8 * dx);
        T a, b;
        cx<T> gg;
        if (rl == 2) {
          // one pair: lane group g of 8 sums Re(conj(u) v) for (u, v) =
          // (x_0, x_0), (x_1, x_1), (x_0, x_1), (x_0, -i x_1) (rows 2, 3 are idle)
          const cx<T> u0 = shcx(x, j), u1 = shcx(x, 8 + j);
          const cx<T> u = p == 1 ? u1 : u0;
          const cx<T> v = p == 0 ? u0 : (p == 3 ? mk<T>(u1.im, -u1.re) : u1);
          const T s8 = sum8(j < c ? fma(u.re, v.re, u.im * v.im) : (T)0);
          a = shidx(s8, 0);
          b = shidx(s8, 8);
          gg = mk<T>(shidx(s8, 16), shidx(s8, 24));
          own2 = p == 0 ? a : b;
        } else {
          const cx<T> xp = isP ? x : y, xq = isP ? y : x;
          const cx<T> xm = j < c ? x : zero;
          const cx<T> g = j < c ? cmacc(zero, xp, xq) : zero;
          const T r4 = sum8x4(abs2(xm), g.re, g.im, (T)0, j);
          a = shidx(r4, lp);
          b = shidx(r4, lq);
          gg = mk<T>(shidx(r4, lp + 2), shidx(r4, lp + 4));
          own2 = isP ? a : b;
        }
        T cc, sre, sim;
        bool small = false;
        const bool rot = p < rl && q < rl && jacobi_rotation<T>(a, b, gg, K<T>::jtolf(), skip2, cc, sre, sim, &small);
        if (rot) {
          // row p: c x_p - conj(s) x_q ; row q: c x_q + s x_p
          const cx<T> coef = isP ? mk<T>(-sre, sim) : mk<T>(sre, sim);
          x = cmac(cscale(x, cc), coef, y);
        }
        rotated = rotated || rot;
        if (rl == 2 && __any_sync(0xffffffffu, rot && small)) done_early = true;
      }
      if (!__any_sync(0xffffffffu, rotated) || done_early) {
        sw = sweep + 1;
        break;
      }
    }
  }
  // sigma_p^2 (rows are orthogonal): the last sweep's Gram diagonal when it
  // rotated nothing, else summed afresh; ranks, rank rule
  const T sp = (sw > 0 && !done_early) ? (row ? own2 : (T)0) : sum8(inM ? abs2(x) : (T)0);
  const T s0 = shidx(sp, 0), s1 = shidx(sp, 8), s2 = shidx(sp, 16), s3 = shidx(sp, 24);
  int rk[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const T su = pick4(s0, s1, s2, s3, u);
    int r = 0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const T sv = pick4(s0, s1, s2, s3, v);
      r += (v < rl && v != u && (nn_gt(sv, su) || (nn_eq(sv, su) && v < u))) ? 1 : 0;
    }
    rk[u] = r;
  }
  int perm[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int who = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) who = (u < rl && rk[u] == t) ? u : who;
    perm[t] = who;
  }
  const T smax = pick4(s0, s1, s2, s3, perm[0]);
  const T fr = fmax(B.tmisc[1], rank_floor(B, rl, c));
  const T thr2 = fr * fr * smax;
  int k = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) k += (u < rl && nn_gt(pick4(s0, s1, s2, s3, u), thr2)) ? 1 : 0;
  if (k < 1) k = 1;
  if (k > d.chi_max) k = d.chi_max;
  const bool over = k > d.chicap;
  if (over) k = d.chicap;
  if (lane == 0) {
    if (sw < 0) set_status<T>(B.misc, kDevNoConv);
    if (over) set_status<T>(B.misc, kDevCapacity);
    const int swc = sw < 0 ? d.max_sweeps : sw;
    B.misc[1] = max(B.misc[1], swc);
    B.misc[2] += swc;
    B.misc[3] += 1;
    B.misc[4] = k;
    B.chi[l] = k;
    if (k < rl) {  // discarded weight, summed in rank order
      T tot = 0, kept = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (t < rl) {
          const T st_ = pick4(s0, s1, s2, s3, perm[t]);
          tot += st_;
          if (t < k) kept += st_;
        }
      }
      if (tot > (T)0 && kept != tot) B.tmisc[2] += (tot - kept) / tot;
    }
  }
  // outputs (all reads of site l and US happened before the shuffles above)
  __syncwarp();
  const int myrank = pick4(rk[0], rk[1], rk[2], rk[3], p);
  if (row && myrank < k) {
    const T inv = rsqrt(sp);
    if (inM) {
      st_site(A + myrank * c + j, cscale(x, inv), B.key(l, 1), myrank * c + j);
    } else if (inU) {
      const T sg = sp * inv;  // sigma = sigma^2 / sigma
      B.US[(j - c) * k + myrank] = mk<T>(x.re * sg, -(x.im * sg));
    }
  }
}
