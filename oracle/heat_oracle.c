/*
 * heat_oracle.c -- the CPU oracle for the periodic 1D heat stencil.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  The CUDA library
 * shares no code, header, table or constant with it, and never calls it.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math (no contraction into FMA, so
 * every operation below is one IEEE binary64 operation rounded to nearest-even,
 * in exactly the order written).
 *
 * The method (paper, Section 2 "Model problem"):
 *   Eq. 1   u_t = alpha * u_xx on a loop 0 <= x < L, periodic u(t,x) = u(t,L+x).
 *   grid    x_i = i*h, i = 0..N-1, second-order central differences in space.
 *   Eq. 2   forward Euler in time:
 *             u(t+dt, x_i) = u(t,x_i) + dt*alpha*(u_{i-1} - 2 u_i + u_{i+1}) / h^2
 *           The printed denominator is "2h"; second-order differencing of u_xx
 *           has h^2 there, and that is the reading taken here (coefficient
 *           r = k*dt/dx^2 with k = alpha, dx = h).
 *   IC      u(0, x_i) = x_i (supplied by the caller through the input array).
 *   Parallel algorithm (Section 2, last paragraph): threads each apply Eq. 2 to
 *           a local segment; single-producer single-consumer queues carry the
 *           ghost zones between neighbouring segments.
 *
 * Reading of the operation order (the paper states none):
 *   v[i] = u[i] + r * ((u[i-1] - 2.0*u[i]) + u[i+1])
 * evaluated left to right, each operation rounded once.  The "fma" variant is
 *   v[i] = fma(r, fma(-2.0, u[i], u[i-1]) + u[i+1], u[i]).
 *
 * Parity status: every function here is pinned by tests against mathematics
 * (exact rational arithmetic, conservation, Fourier-mode decay, the maximum
 * principle, special cases); see tests/test_oracle.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Coefficient of Eq. 2 with the h^2 reading: r = (k*dt)/(dx*dx). */
double heat_oracle_r(double k, double dt, double dx) { return (k * dt) / (dx * dx); }

/* One forward-Euler step of Eq. 2 over the whole periodic ring (the
 * unsegmented "synchronous" form the paper describes for Chapel, Section 3.1).
 * Ghosts are at the same time level as the interior. */
static void step_plain(const double *u, double *v, int64_t N, double r) {
  for (int64_t i = 0; i < N; ++i) {
    double ul = u[(i - 1 + N) % N];
    double ur = u[(i + 1) % N];
    v[i] = u[i] + r * ((ul - 2.0 * u[i]) + ur);
  }
}

static void step_fma(const double *u, double *v, int64_t N, double r) {
  for (int64_t i = 0; i < N; ++i) {
    double ul = u[(i - 1 + N) % N];
    double ur = u[(i + 1) % N];
    v[i] = fma(r, fma(-2.0, u[i], ul) + ur, u[i]);
  }
}

/* nt steps of Eq. 2 on a ring of N points.  u holds u^0 on entry and u^nt on
 * return; work is caller-provided scratch of N doubles.  fma selects the
 * fused reading.  Returns 0, or -1 on bad sizes. */
int heat_oracle_run(double *u, double *work, int64_t N, double r, int64_t nt, int fma_form) {
  if (N < 1 || nt < 0) return -1;
  double *a = u, *b = work;
  for (int64_t s = 0; s < nt; ++s) {
    if (fma_form) step_fma(a, b, N, r); else step_plain(a, b, N, r);
    double *t = a; a = b; b = t;
  }
  if (a != u) memcpy(u, a, (size_t)N * sizeof(double));
  return 0;
}

/* ---- The segmented algorithm of Section 2: np segments of nx points, each
 * with one ghost cell per side, ghost values carried by SPSC FIFO queues.
 * Run single-threaded here: every segment pushes its two edge values, then
 * every segment pops its two ghosts and applies Eq. 2 locally.  The result is
 * the same per point as the unsegmented ring (same operation on the same
 * operands), which the tests check bitwise. */
typedef struct { double buf[4]; int head, tail; } spsc_fifo; /* capacity 4 > the 1 in flight */

static void fifo_push(spsc_fifo *q, double x) { q->buf[q->tail & 3] = x; q->tail++; }
static double fifo_pop(spsc_fifo *q) { double x = q->buf[q->head & 3]; q->head++; return x; }

int heat_oracle_run_segmented(double *u, int64_t nx, int32_t np, double r, int64_t nt) {
  if (nx < 1 || np < 1 || nt < 0) return -1;
  const int64_t L = nx + 2; /* local segment: ghost, nx points, ghost */
  double *cur = (double *)malloc(sizeof(double) * (size_t)(L * np));
  double *nxt = (double *)malloc(sizeof(double) * (size_t)(L * np));
  /* from_right[p]: the queue segment p consumes its right ghost from (the
   * producer is p+1); from_left[p]: its left ghost (the producer is p-1). */
  spsc_fifo *from_right = (spsc_fifo *)calloc((size_t)np, sizeof(spsc_fifo));
  spsc_fifo *from_left = (spsc_fifo *)calloc((size_t)np, sizeof(spsc_fifo));
  if (!cur || !nxt || !from_right || !from_left) {
    free(cur); free(nxt); free(from_right); free(from_left);
    return -2;
  }
  for (int32_t p = 0; p < np; ++p)
    memcpy(cur + p * L + 1, u + (int64_t)p * nx, (size_t)nx * sizeof(double));
  for (int64_t s = 0; s < nt; ++s) {
    for (int32_t p = 0; p < np; ++p) {
      int32_t left = (p - 1 + np) % np, right = (p + 1) % np;
      fifo_push(&from_right[left], cur[p * L + 1]);   /* my first point: left's right ghost */
      fifo_push(&from_left[right], cur[p * L + nx]);  /* my last point: right's left ghost */
    }
    for (int32_t p = 0; p < np; ++p) {
      double *c = cur + p * L, *n = nxt + p * L;
      c[0] = fifo_pop(&from_left[p]);
      c[nx + 1] = fifo_pop(&from_right[p]);
      for (int64_t j = 1; j <= nx; ++j) n[j] = c[j] + r * ((c[j - 1] - 2.0 * c[j]) + c[j + 1]);
    }
    double *t = cur; cur = nxt; nxt = t;
  }
  for (int32_t p = 0; p < np; ++p)
    memcpy(u + (int64_t)p * nx, cur + p * L + 1, (size_t)nx * sizeof(double));
  free(cur); free(nxt); free(from_right); free(from_left);
  return 0;
}

/* ---- Light cone: u^nt[g] depends only on u^0[g-nt .. g+nt] (mod N).  Copy
 * that window and apply Eq. 2 on a shrinking line, same operation order.
 * out[q] = u^nt[idx[q]] for q = 0..nq-1; work holds 2*nt+1 doubles. */
int heat_oracle_cone(const double *u0, int64_t N, double r, int64_t nt, const int64_t *idx,
                     int64_t nq, double *out, int fma_form) {
  if (N < 1 || nt < 0) return -1;
  const int64_t W = 2 * nt + 1;
  double *w = (double *)malloc(sizeof(double) * (size_t)W);
  if (!w) return -2;
  for (int64_t q = 0; q < nq; ++q) {
    int64_t g = idx[q];
    if (g < 0 || g >= N) { free(w); return -1; }
    for (int64_t j = 0; j < W; ++j) {
      int64_t src = ((g - nt + j) % N + N) % N;
      w[j] = u0[src];
    }
    /* after step s the valid entries are j = s .. W-1-s; update in place from
     * left to right keeping the old left neighbour in a temporary */
    for (int64_t s = 1; s <= nt; ++s) {
      double prev = w[s - 1];
      for (int64_t j = s; j <= W - 1 - s; ++j) {
        double c = w[j];
        double v = fma_form ? fma(r, fma(-2.0, c, prev) + w[j + 1], c)
                            : c + r * ((prev - 2.0 * c) + w[j + 1]);
        prev = c;
        w[j] = v;
      }
    }
    out[q] = w[nt];
  }
  free(w);
  return 0;
}

/* ---- FP32 storage with a compensated update (the library's reduced-precision
 * form; the paper has no precision study, so this follows the library's own
 * definition).  The state is stored as float.  Time is cut into blocks of T
 * steps (the last block may be shorter).  At the start of a block each point
 * carries hi = stored value, lo = 0; every step of the block does
 *     d   = ((hl - 2 h) + hr) + ((ll - 2 l) + lr)
 *     inc = rf * d
 *     (s, e) = TwoSum(h, inc)           (Knuth's six-operation exact sum)
 *     h' = s,  l' = l + e
 * and at the end of the block the stored value is RN(h + l).  All operations
 * are binary32, rounded to nearest-even, in the order written. */
static void two_sum(float a, float b, float *s, float *e) {
  float ss = a + b;
  float bb = ss - a;
  float ee = (a - (ss - bb)) + (b - bb);
  *s = ss; *e = ee;
}

int heat_oracle_run_f32c(float *u, int64_t N, float rf, int64_t nt, int64_t T) {
  if (N < 1 || nt < 0 || T < 1) return -1;
  float *h = (float *)malloc(sizeof(float) * (size_t)N), *l = (float *)malloc(sizeof(float) * (size_t)N);
  float *h2 = (float *)malloc(sizeof(float) * (size_t)N), *l2 = (float *)malloc(sizeof(float) * (size_t)N);
  if (!h || !l || !h2 || !l2) { free(h); free(l); free(h2); free(l2); return -2; }
  int64_t done = 0;
  while (done < nt) {
    int64_t steps = nt - done < T ? nt - done : T;
    for (int64_t i = 0; i < N; ++i) { h[i] = u[i]; l[i] = 0.0f; }
    for (int64_t s = 0; s < steps; ++s) {
      for (int64_t i = 0; i < N; ++i) {
        int64_t im = (i - 1 + N) % N, ip = (i + 1) % N;
        float dh = (h[im] - 2.0f * h[i]) + h[ip];
        float dl = (l[im] - 2.0f * l[i]) + l[ip];
        float d = dh + dl;
        float inc = rf * d;
        float sum, err;
        two_sum(h[i], inc, &sum, &err);
        h2[i] = sum;
        l2[i] = l[i] + err;
      }
      float *t = h; h = h2; h2 = t;
      t = l; l = l2; l2 = t;
    }
    for (int64_t i = 0; i < N; ++i) u[i] = h[i] + l[i];
    done += steps;
  }
  free(h); free(l); free(h2); free(l2);
  return 0;
}

/* ---- Diagnostics: plain left-to-right FP64 sum (conservation of sum(u) on
 * the ring is exact in real arithmetic for Eq. 2). */
double heat_oracle_sum(const double *u, int64_t N) {
  double s = 0.0;
  for (int64_t i = 0; i < N; ++i) s += u[i];
  return s;
}
