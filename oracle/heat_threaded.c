/*
 * heat_threaded.c -- the paper's parallel algorithm on the host's cores.
 *
 * TEST INFRASTRUCTURE AND CPU BASELINE ONLY.  Like heat_oracle.c, only the
 * test suite and the benchmark's CPU-baseline leg load it; the CUDA library
 * shares nothing with it.  Build: gcc -O2 -ffp-contract=off -fno-fast-math
 * -pthread.
 *
 * Section 2, last paragraph: the ring of np*nx points is cut into np segments
 * of nx points; each segment is advanced by its own thread, which keeps a
 * local copy with one ghost cell per side and, every step, sends its first
 * point to the left neighbour and its last point to the right neighbour
 * through single-producer single-consumer queues, then takes its two ghosts
 * from its own incoming queues (Section 3 describes the per-language queues;
 * the C++ one is a queue guarded by a mutex and a condition variable, which is
 * what this file uses).  Each point is updated with Eq. 2 in the same
 * operation order as heat_oracle.c, so the result equals the oracle's bitwise
 * (tests/test_oracle.py checks it).
 *
 * A thread can run at most one step ahead of a neighbour (it needs that
 * neighbour's edge value of the current step before it can finish the step),
 * so at most two values are ever queued on an edge; the queues hold four.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double buf[4];
  int head, tail;  /* pop at head, push at tail; count = tail - head */
  pthread_mutex_t mu;
  pthread_cond_t cv;
} queue_t;

static void q_init(queue_t *q) {
  q->head = q->tail = 0;
  pthread_mutex_init(&q->mu, NULL);
  pthread_cond_init(&q->cv, NULL);
}

static void q_free(queue_t *q) {
  pthread_mutex_destroy(&q->mu);
  pthread_cond_destroy(&q->cv);
}

static void q_push(queue_t *q, double x) {
  pthread_mutex_lock(&q->mu);
  while (q->tail - q->head == 4) pthread_cond_wait(&q->cv, &q->mu);
  q->buf[q->tail & 3] = x;
  q->tail++;
  pthread_cond_broadcast(&q->cv);
  pthread_mutex_unlock(&q->mu);
}

static double q_pop(queue_t *q) {
  pthread_mutex_lock(&q->mu);
  while (q->tail == q->head) pthread_cond_wait(&q->cv, &q->mu);
  const double x = q->buf[q->head & 3];
  q->head++;
  pthread_cond_broadcast(&q->cv);
  pthread_mutex_unlock(&q->mu);
  return x;
}

/* Start gate: workers wait until every thread exists (go = 1), or leave at
 * once if one could not be created (go = -1). */
typedef struct {
  pthread_mutex_t mu;
  pthread_cond_t cv;
  int go;
} gate_t;

typedef struct {
  gate_t *gate;
  double *cur, *nxt;      /* local arrays of nx + 2: ghost, nx points, ghost */
  int64_t nx, nt;
  double r;
  queue_t *from_left;     /* this segment's left ghosts (pushed by the left neighbour) */
  queue_t *from_right;    /* its right ghosts (pushed by the right neighbour) */
  queue_t *to_left;       /* the left neighbour's from_right */
  queue_t *to_right;      /* the right neighbour's from_left */
} seg_t;

static void *segment_worker(void *arg) {
  seg_t *g = (seg_t *)arg;
  pthread_mutex_lock(&g->gate->mu);
  while (g->gate->go == 0) pthread_cond_wait(&g->gate->cv, &g->gate->mu);
  const int go = g->gate->go;
  pthread_mutex_unlock(&g->gate->mu);
  if (go < 0) return NULL;
  const int64_t nx = g->nx;
  for (int64_t s = 0; s < g->nt; ++s) {
    double *c = g->cur, *n = g->nxt;
    q_push(g->to_left, c[1]);
    q_push(g->to_right, c[nx]);
    c[0] = q_pop(g->from_left);
    c[nx + 1] = q_pop(g->from_right);
    for (int64_t j = 1; j <= nx; ++j) n[j] = c[j] + g->r * ((c[j - 1] - 2.0 * c[j]) + c[j + 1]);
    g->cur = n;
    g->nxt = c;
  }
  return NULL;
}

/* nt steps of Eq. 2 on the ring u (np*nx points, global order), one thread per
 * segment.  Returns 0, -1 on bad sizes, -2 if memory or a thread could not be
 * had. */
int heat_threaded_run(double *u, int64_t nx, int32_t np, double r, int64_t nt) {
  if (nx < 1 || np < 1 || nt < 0) return -1;
  const int64_t L = nx + 2;
  double *mem = (double *)malloc(sizeof(double) * (size_t)(2 * L * np));
  seg_t *seg = (seg_t *)calloc((size_t)np, sizeof(seg_t));
  queue_t *qin_l = (queue_t *)calloc((size_t)np, sizeof(queue_t));
  queue_t *qin_r = (queue_t *)calloc((size_t)np, sizeof(queue_t));
  pthread_t *th = (pthread_t *)calloc((size_t)np, sizeof(pthread_t));
  int rc = 0;
  if (!mem || !seg || !qin_l || !qin_r || !th) {
    rc = -2;
    goto out;
  }
  for (int32_t p = 0; p < np; ++p) {
    q_init(&qin_l[p]);
    q_init(&qin_r[p]);
  }
  for (int32_t p = 0; p < np; ++p) {
    const int32_t left = (p - 1 + np) % np, right = (p + 1) % np;
    seg[p].cur = mem + 2 * L * p;
    seg[p].nxt = seg[p].cur + L;
    memcpy(seg[p].cur + 1, u + (int64_t)p * nx, (size_t)nx * sizeof(double));
    seg[p].nx = nx;
    seg[p].nt = nt;
    seg[p].r = r;
    seg[p].from_left = &qin_l[p];
    seg[p].from_right = &qin_r[p];
    seg[p].to_left = &qin_r[left];
    seg[p].to_right = &qin_l[right];
  }
  gate_t gate;
  pthread_mutex_init(&gate.mu, NULL);
  pthread_cond_init(&gate.cv, NULL);
  gate.go = 0;
  for (int32_t p = 0; p < np; ++p) seg[p].gate = &gate;
  int32_t started = 0;
  for (; started < np; ++started)
    if (pthread_create(&th[started], NULL, segment_worker, &seg[started]) != 0) break;
  pthread_mutex_lock(&gate.mu);
  gate.go = started == np ? 1 : -1;  /* all or none of the segments run */
  pthread_cond_broadcast(&gate.cv);
  pthread_mutex_unlock(&gate.mu);
  for (int32_t p = 0; p < started; ++p) pthread_join(th[p], NULL);
  pthread_mutex_destroy(&gate.mu);
  pthread_cond_destroy(&gate.cv);
  if (started == np) {
    for (int32_t p = 0; p < np; ++p) memcpy(u + (int64_t)p * nx, seg[p].cur + 1, (size_t)nx * sizeof(double));
  } else {
    rc = -2;
  }
  for (int32_t p = 0; p < np; ++p) {
    q_free(&qin_l[p]);
    q_free(&qin_r[p]);
  }
out:
  free(mem);
  free(seg);
  free(qin_l);
  free(qin_r);
  free(th);
  return rc;
}
