// Whole MIXED solves of small 1D problems in one CTA (Algorithm 1 with the residual-correction
// form, every sweep, and the stopping rule): the iterate, the time tile and the spatial tile live
// in shared memory, so a solve is one launch whose sweeps are separated by block barriers only.
// A problem of a few thousand space-time unknowns (the 1D heat problem of 63 points and 64
// levels) takes several microseconds per kernel in the multi-kernel sweep, nearly all of it
// launch and memory latency; here the same arithmetic runs back to back on one SM.
//
// Per sweep, identical in arithmetic to the multi-kernel MIXED sweep:
//   1. r = F_hat - K U in double-float (BDF band with zero history before level 0, the 3-point
//      stencil with power-of-two weight 1/h^2), scaled by kappa^{n/N}, into the time tile
//      (point m in complex column m mod Ct, real part for m < Ct, imaginary part otherwise);
//   2. forward FFT along time; the two half spectra of each column separated;
//   3. for each frequency j <= N/2 (in batches of Cs lines, Cs dividing N/2, and the line j = N/2
//      alone): sine transform of the odd extension, divide by 2(M+1) (sigma_j + lambda_p), inverse
//      transform -- the shifted systems (sigma_j + A_h) q_j = h_j of Algorithm 1, step 2;
//   4. the spectra recombined, inverse FFT along time, unscaled by kappa^{-n/N}/N;
//   5. U += c in double-float, the norms of c and U (FP32 partials), the stopping rule.
#include "ff.cuh"
#include "fft.cuh"
#include "pint_internal.h"

namespace pint {

namespace {

__host__ __device__ inline size_t small_align(size_t x) { return (x + 15) & ~(size_t)15; }

struct SmallLayout {
  size_t U, Fh, Xt, Xs, twt, twx, pt, px, s, is, sig, lam, red, total;
};

// byte offsets of the shared-memory carve-up
__host__ __device__ inline SmallLayout small_layout(int N, int M, int Ct, int L, int Cs) {
  SmallLayout l;
  size_t o = 0;
  l.U = o;   o = small_align(o + sizeof(float2) * (size_t)N * M);          // iterate (hi, lo)
  l.Fh = o;  o = small_align(o + sizeof(float2) * (size_t)N * M);          // F_hat split (hi, lo)
  l.Xt = o;  o = small_align(o + sizeof(float2) * (size_t)N * Ct);         // time tile [N][Ct]
  l.Xs = o;  o = small_align(o + sizeof(float2) * (size_t)L * (Cs + 1));   // spatial tile [L][Cs+1]
  l.twt = o; o = small_align(o + sizeof(float2) * (size_t)N);
  l.twx = o; o = small_align(o + sizeof(float2) * (size_t)L);
  l.pt = o;  o = small_align(o + sizeof(unsigned short) * (size_t)N);
  l.px = o;  o = small_align(o + sizeof(unsigned short) * (size_t)L);
  l.s = o;   o = small_align(o + sizeof(float) * (size_t)N);
  l.is = o;  o = small_align(o + sizeof(float) * (size_t)N);
  l.sig = o; o = small_align(o + sizeof(float2) * (size_t)(N / 2 + 1));
  l.lam = o; o = small_align(o + sizeof(float) * (size_t)M);
  l.red = o; o = small_align(o + sizeof(float) * 64 + sizeof(int) * 4);
  l.total = o;
  return l;
}

// stop_decision in FP32 (one thread decides while the block waits at a barrier, and FP64
// arithmetic runs at ~1/70 of the FP32 rate; a stopping rule needs no more than FP32)
__device__ __forceinline__ bool stop_decision_f(int m, float upd, float prev, float tol, float q_floor) {
  if (m == 1) return upd <= 0.01f * tol;
  const float q = prev > 0.f ? upd / prev : 0.f;
  const float qh = q > q_floor ? q : q_floor;
  if (qh < 1.f) return upd * qh / (1.f - qh) <= tol;
  return upd <= tol;
}

__global__ void __launch_bounds__(kSmallThreads) k_small_solve(SmallArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = a.N, M = a.M, Ct = a.Ct, logCt = a.logCt, L = a.L, Cs = a.Cs, logCs = a.logCs;
  const int J = N / 2 + 1, n = M, logP = logCt + 1;
  const SmallLayout lay = small_layout(N, M, Ct, L, Cs);
  float2* U = reinterpret_cast<float2*>(sm + lay.U);
  float2* Fh = reinterpret_cast<float2*>(sm + lay.Fh);
  float2* Xt = reinterpret_cast<float2*>(sm + lay.Xt);
  float* Xtf = reinterpret_cast<float*>(Xt);
  float2* Xs = reinterpret_cast<float2*>(sm + lay.Xs);
  float2* twt = reinterpret_cast<float2*>(sm + lay.twt);
  float2* twx = reinterpret_cast<float2*>(sm + lay.twx);
  unsigned short* pt = reinterpret_cast<unsigned short*>(sm + lay.pt);
  unsigned short* px = reinterpret_cast<unsigned short*>(sm + lay.px);
  float* s = reinterpret_cast<float*>(sm + lay.s);
  float* is = reinterpret_cast<float*>(sm + lay.is);
  float2* sig = reinterpret_cast<float2*>(sm + lay.sig);
  float* lam = reinterpret_cast<float*>(sm + lay.lam);
  float* red = reinterpret_cast<float*>(sm + lay.red);   // [2][32] warp partials
  int* flag = reinterpret_cast<int*>(red + 64);
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;

  for (int i = tid; i < N; i += nth) {
    twt[i] = a.tw_t[i];
    s[i] = a.s[i];
    is[i] = a.inv_s[i];
  }
  for (int i = tid; i < L; i += nth) twx[i] = a.tw_x[i];
  for (int j = tid; j < J; j += nth) sig[j] = a.sigma[j];
  for (int i = tid; i < M; i += nth) lam[i] = a.lam[i];
  fft_perm_table(pt, N);
  fft_perm_table(px, L);
  // U_0 (v on every level, or the caller's guess) and F_hat split into double-float once, in
  // batches of 8 independent loads per thread
  const int NM = N * M;
  for (int e0 = tid; e0 < NM; e0 += 8 * nth) {
    double f[8], u[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = e0 + t * nth;
      f[t] = e < NM ? a.F[e] : 0.0;
      u[t] = e < NM ? (a.v ? a.v[e % M] : a.U[e]) : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = e0 + t * nth;
      if (e < NM) {
        const ff fx = ff_split_trunc(f[t]);
        Fh[e] = make_float2(fx.hi, fx.lo);
        const ff ux = ff_from_double(u[t]);
        U[e] = make_float2(ux.hi, ux.lo);
      }
    }
  }
  __syncthreads();

  const float gx = a.gx;
  const float scale = (float)(2 * (M + 1));
  const float tolf = (float)a.tol, qfl = (float)a.q_floor;
  float prev = 0.f, upd = 0.f;
  int m_done = 0;
  for (int sweep = 1; sweep <= a.max_sweeps; ++sweep) {
    // 1. residual into the time tile
#pragma unroll 2
    for (int e = tid; e < (N << logP); e += nth) {
      const int i = e >> logP, q = e & ((1 << logP) - 1);
      float val = 0.f;
      if (q < M) {
        const int idx = i * M + q;
        ff_acc A;
        const float2 fh = Fh[idx];
        A.init(ff{fh.x, fh.y});
        const float2 c = U[idx];
        A.fma_term(ff{a.c_hi[0], a.c_lo[0]}, ff{c.x, c.y}, -1.f);
#pragma unroll
        for (int t = 1; t <= kMaxK; ++t) {
          if (t <= a.k && i - t >= 0) {
            const float2 h = U[idx - t * M];
            A.fma_term(ff{a.c_hi[t], a.c_lo[t]}, ff{h.x, h.y}, -1.f);
          }
        }
        const float2 w = q > 0 ? U[idx - 1] : make_float2(0.f, 0.f);
        const float2 o = q < M - 1 ? U[idx + 1] : make_float2(0.f, 0.f);
        float bx, ex;
        two_sum(w.x, o.x, bx, ex);
        A.add_hi(gx * bx);
        A.sl += gx * (ex + (w.y + o.y));
        val = A.value() * s[i];
      }
      Xtf[2 * (i * Ct + (q & (Ct - 1))) + (q >> logCt)] = val;
    }
    __syncthreads();
    fft_forward(Xt, Ct, logCt, N, twt);

    // 2./3./4. per batch of frequencies: separate, sine-transform solve, recombine. Cs divides
    // N/2, so the lines j = 0..N/2-1 fill whole batches of Cs and the last line, j = N/2, is a
    // batch of its own (no padding columns).
    for (int j0 = 0; j0 < J;) {
      const int cs = j0 + Cs <= J - 1 ? Cs : 1, logcs = cs == Cs ? logCs : 0, ld = cs + 1;
      for (int e = tid; e < (n << logcs); e += nth) {
        const int cc = e & (cs - 1), i = e >> logcs, j = j0 + cc;
        const int col = i & (Ct - 1);
        const float2 zj = Xt[pt[j] * Ct + col], zn = Xt[pt[(N - j) & (N - 1)] * Ct + col];
        const float2 v = (i >> logCt) ? make_float2(0.5f * (zj.y + zn.y), -0.5f * (zj.x - zn.x))  // B: (Z_j - conj Z_{N-j}) / 2i
                                      : make_float2(0.5f * (zj.x + zn.x), 0.5f * (zj.y - zn.y));  // A: (Z_j + conj Z_{N-j}) / 2
        Xs[(i + 1) * ld + cc] = v;
        Xs[(L - 1 - i) * ld + cc] = make_float2(-v.x, -v.y);
      }
      for (int cc = tid; cc < cs; cc += nth) {
        Xs[cc] = make_float2(0.f, 0.f);
        Xs[(n + 1) * ld + cc] = make_float2(0.f, 0.f);
      }
      __syncthreads();
      fft_forward(Xs, ld, logcs, L, twx);
      for (int e = tid; e < ((n + 2) << logcs); e += nth) {
        const int cc = e & (cs - 1), p = e >> logcs, j = j0 + cc;
        const int pos = px[p] * ld + cc;
        if (p == 0 || p == n + 1) {
          Xs[pos] = make_float2(0.f, 0.f);
          continue;
        }
        const float dx = (sig[j].x + lam[p - 1]) * scale, dy = sig[j].y * scale;
        const float inv = __frcp_rn(dx * dx + dy * dy);
        const float2 qd = make_float2(dx * inv, dy * inv);
        const int pos2 = px[L - p] * ld + cc;
        Xs[pos] = cmulc(Xs[pos], qd);
        Xs[pos2] = cmulc(Xs[pos2], qd);
      }
      __syncthreads();
      fft_inverse(Xs, ld, logcs, L, twx);
      for (int e = tid; e < (cs << logCt); e += nth) {
        const int col = e & (Ct - 1), cc = e >> logCt, j = j0 + cc;
        const float2 A = col < n ? Xs[(col + 1) * ld + cc] : make_float2(0.f, 0.f);
        const float2 B = col + Ct < n ? Xs[(col + Ct + 1) * ld + cc] : make_float2(0.f, 0.f);
        Xt[pt[j] * Ct + col] = make_float2(A.x - B.y, A.y + B.x);                      // A + iB
        if (j > 0 && j < N / 2) Xt[pt[N - j] * Ct + col] = make_float2(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
      }
      __syncthreads();
      j0 += cs;
    }
    fft_inverse(Xt, Ct, logCt, N, twt);

    // 5. update and norms
    float sc = 0.f, su = 0.f;
    for (int e = tid; e < (N << logP); e += nth) {
      const int i = e >> logP, q = e & ((1 << logP) - 1);
      if (q >= M) continue;
      const float c = Xtf[2 * (i * Ct + (q & (Ct - 1))) + (q >> logCt)] * is[i];
      const float2 u0 = U[i * M + q];
      const ff u = ff_add_f(ff{u0.x, u0.y}, c);
      U[i * M + q] = make_float2(u.hi, u.lo);
      sc = fmaf(c, c, sc);
      su = fmaf(u.hi, u.hi, su);
    }
    for (int o = 16; o > 0; o >>= 1) {
      sc += __shfl_down_sync(0xffffffffu, sc, o);
      su += __shfl_down_sync(0xffffffffu, su, o);
    }
    if (lane == 0) { red[warp] = sc; red[32 + warp] = su; }
    __syncthreads();
    if (tid == 0) {
      float c2 = 0.f, u2 = 0.f;
      for (int w = 0; w < (nth >> 5); ++w) { c2 += red[w]; u2 += red[32 + w]; }
      upd = u2 > 0.f ? sqrtf(c2 / u2) : sqrtf(c2);
      flag[0] = stop_decision_f(sweep, upd, prev, tolf, qfl) ? 1 : 0;
      prev = upd;
    }
    m_done = sweep;
    __syncthreads();
    if (flag[0]) break;
  }

  for (int e = tid; e < N * M; e += nth) a.U[e] = ff_to_double(ff{U[e].x, U[e].y});
  if (tid == 0) {
    SolveCtl* c = a.ctl;
    c->tol = a.tol;
    c->q_floor = a.q_floor;
    c->max_sweeps = a.max_sweeps;
    c->m = m_done;
    c->prev = prev;
    c->upd = upd;
    c->done = flag[0];
  }
}

}  // namespace

size_t small_smem(int N, int M, int Ct, int L, int Cs) { return small_layout(N, M, Ct, L, Cs).total; }

cudaError_t launch_small_solve(const SmallArgs& a, cudaStream_t st) {
  const size_t sm = small_smem(a.N, a.M, a.Ct, a.L, a.Cs);
  cudaError_t e = cudaFuncSetAttribute(k_small_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  prof_begin("small_solve_ff", st);
  k_small_solve<<<1, kSmallThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

}  // namespace pint
