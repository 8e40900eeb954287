/*
 * mpf_oracle.c -- scalar reference for the MSV and SSV byte filters.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA scan
 * library is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * What it computes (one profile, many sequences, one pass per sequence,
 * no blocking, no vectorisation, every byte saturation written out):
 *
 *   MSV (Sec. 2.1: ungapped local model with multiple hits, Insert/Delete
 *   states pruned, M->M transition treated as probability 1; byte update of
 *   Alg. 2 with its special-state update, following the MSV filter of the
 *   HMMER3 paper cited in Sec. 2.1):
 *
 *     dp[0..M] = 0, xJ = 0, xB = sat(base - (t + tbm))
 *     for each residue x_i:
 *        for k = 1..M (previous-row values on the right-hand side, dp[0] = 0):
 *           dp[k] = sat( sat( max(dp[k-1], xB) + bias ) - cost[x_i][k] )
 *        xE = max_k dp[k]
 *        if xE >= 255 - bias  ->  overflow: raw = 255, flag = 1, nat = +inf
 *        xJ = max(xJ, sat(xE - tec))
 *        xB = sat(max(base, xJ) - (t + tbm))
 *     raw = xJ, nat = (float)(xJ - t - base) / scale - 3
 *
 *   SSV (Sec. 2.1: the MSV model with the J state removed; byte update of
 *   Alg. 7, read in the unsigned offset form r = stored - 0x80 so that the
 *   floor 0 is the "restart the segment" value and the cap is 255):
 *
 *     r[0..M] = 0, R = 0
 *     for each residue x_i, for k = 1..M (previous-row values, r[0] = 0):
 *        r[k] = min(255, max(0, r[k-1] + bias - cost[x_i][k]))
 *        R = max(R, r[k])
 *     raw = R, flag = (R == 255),
 *     nat = flag ? +inf : (float)(R - tbm - tec - 2 t) / scale - 3
 *
 *   with sat(v) = min(255, max(0, v)), t = tjb(L) taken from the per-length
 *   table (last entry for longer sequences) or the fixed byte, and residue
 *   codes x >= K scoring with cost 255 at every node.
 *
 * The nat arithmetic is IEEE single precision: int -> float conversion, one
 * division, one subtraction, in that order (build with -ffp-contract=off).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int M, K;
  const uint8_t *cost; /* K x M, row-major [x][k-1] */
  uint8_t bias, tbm, tec, tjb_fixed, base;
  const uint8_t *tjb_by_len; /* nullable */
  uint32_t n_tjb;
  float scale;
} oracle_profile;

static int sat8(int v) { return v < 0 ? 0 : (v > 255 ? 255 : v); }

static int cost_of(const oracle_profile *p, int x, int k /* 1..M */) {
  if (x >= p->K) return 255;
  return p->cost[(size_t)x * (size_t)p->M + (size_t)(k - 1)];
}

static int tjb_for_length(const oracle_profile *p, uint32_t L) {
  if (p->tjb_by_len == NULL || p->n_tjb == 0) return p->tjb_fixed;
  return p->tjb_by_len[L < p->n_tjb ? L : p->n_tjb - 1];
}

/* One MSV sequence.  prev/cur are caller scratch of M+1 ints. */
static void msv_one(const oracle_profile *p, const uint8_t *seq, uint32_t L,
                    int *prev, int *cur, uint8_t *raw, uint8_t *flag, float *nat) {
  const int M = p->M;
  const int t = tjb_for_length(p, L);
  const int bias = p->bias;
  int xJ = 0;
  int xB = sat8((int)p->base - (t + (int)p->tbm));
  for (int k = 0; k <= M; ++k) prev[k] = 0;
  for (uint32_t i = 0; i < L; ++i) {
    const int x = seq[i];
    int xE = 0;
    cur[0] = 0;
    for (int k = 1; k <= M; ++k) {
      int from = prev[k - 1] > xB ? prev[k - 1] : xB;   /* M(k-1) or B -> M(k) */
      int v = sat8(from + bias);                        /* add the bias       */
      v = sat8(v - cost_of(p, x, k));                   /* subtract the cost  */
      cur[k] = v;
      if (v > xE) xE = v;                               /* M(k) -> E          */
    }
    if (xE >= 255 - bias) {                             /* saturation reached */
      *raw = 255; *flag = 1; *nat = INFINITY;
      return;
    }
    int xEj = sat8(xE - (int)p->tec);                   /* E -> J             */
    if (xEj > xJ) xJ = xEj;
    int bj = (int)p->base > xJ ? (int)p->base : xJ;     /* N or J -> B        */
    xB = sat8(bj - (t + (int)p->tbm));
    int *sw = prev; prev = cur; cur = sw;
  }
  *raw = (uint8_t)xJ;
  *flag = 0;
  float num = (float)(xJ - t - (int)p->base);
  *nat = num / p->scale - 3.0f;
}

/* One SSV sequence. */
static void ssv_one(const oracle_profile *p, const uint8_t *seq, uint32_t L,
                    int *prev, int *cur, uint8_t *raw, uint8_t *flag, float *nat) {
  const int M = p->M;
  const int t = tjb_for_length(p, L);
  const int bias = p->bias;
  int R = 0;
  for (int k = 0; k <= M; ++k) prev[k] = 0;
  for (uint32_t i = 0; i < L; ++i) {
    const int x = seq[i];
    cur[0] = 0;
    for (int k = 1; k <= M; ++k) {
      int v = prev[k - 1] + bias - cost_of(p, x, k);
      v = sat8(v);
      cur[k] = v;
      if (v > R) R = v;
    }
    int *sw = prev; prev = cur; cur = sw;
  }
  *raw = (uint8_t)R;
  if (R == 255) {
    *flag = 1; *nat = INFINITY;
  } else {
    *flag = 0;
    float num = (float)(R - (int)p->tbm - (int)p->tec - 2 * t);
    *nat = num / p->scale - 3.0f;
  }
}

typedef struct {
  const oracle_profile *p;
  int filter; /* 0 = MSV, 1 = SSV */
  const uint8_t *residues;
  const uint64_t *offsets;
  const uint32_t *lengths;
  const uint64_t *index; /* nullable: sequences to score, else 0..n-1 */
  uint64_t n;
  uint8_t *raw, *flag;
  float *nat;
  uint64_t begin, end;
  int err;
} oracle_job;

static void *oracle_worker(void *arg) {
  oracle_job *j = (oracle_job *)arg;
  int *a = (int *)malloc(sizeof(int) * ((size_t)j->p->M + 1));
  int *b = (int *)malloc(sizeof(int) * ((size_t)j->p->M + 1));
  if (!a || !b) { j->err = 1; free(a); free(b); return NULL; }
  for (uint64_t q = j->begin; q < j->end; ++q) {
    uint64_t s = j->index ? j->index[q] : q;
    const uint8_t *seq = j->residues + j->offsets[s];
    if (j->filter == 0)
      msv_one(j->p, seq, j->lengths[s], a, b, &j->raw[q], &j->flag[q], &j->nat[q]);
    else
      ssv_one(j->p, seq, j->lengths[s], a, b, &j->raw[q], &j->flag[q], &j->nat[q]);
  }
  free(a); free(b);
  return NULL;
}

/*
 * Score sequences with one profile.  All pointers are host pointers.
 *   filter:   0 = MSV, 1 = SSV
 *   cost:     K x M bytes, row-major [x][k-1]
 *   tjb_by_len: nullable per-length tjb table of n_tjb entries
 *   index:    nullable list of n sequence numbers to score (outputs are in
 *             the order of this list); NULL scores sequences 0..n-1
 *   nthreads: worker threads (<= 1: run on the calling thread)
 * Returns 0 on success, 1 on bad arguments, 2 on allocation failure.
 */
int oracle_scan(int filter, int M, int K, const uint8_t *cost, uint8_t bias, uint8_t tbm,
                uint8_t tec, uint8_t tjb_fixed, const uint8_t *tjb_by_len, uint32_t n_tjb,
                float scale, uint8_t base, const uint8_t *residues, const uint64_t *offsets,
                const uint32_t *lengths, const uint64_t *index, uint64_t n, uint8_t *raw,
                uint8_t *flag, float *nat, int nthreads) {
  if (M < 1 || K < 1 || K > 32 || !cost || (filter != 0 && filter != 1)) return 1;
  if (n > 0 && (!residues || !offsets || !lengths || !raw || !flag || !nat)) return 1;
  oracle_profile p = {M, K, cost, bias, tbm, tec, tjb_fixed, base, tjb_by_len, n_tjb, scale};
  if (nthreads < 1) nthreads = 1;
  if ((uint64_t)nthreads > n) nthreads = n > 0 ? (int)n : 1;
  oracle_job *jobs = (oracle_job *)calloc((size_t)nthreads, sizeof(oracle_job));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return 2; }
  /* Contiguous static split: thread w scores list entries [w*chunk, (w+1)*chunk). */
  uint64_t chunk = (n + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
  for (int w = 0; w < nthreads; ++w) {
    jobs[w] = (oracle_job){&p, filter, residues, offsets, lengths, index, n, raw, flag, nat,
                           (uint64_t)w * chunk, (uint64_t)(w + 1) * chunk, 0};
    if (jobs[w].begin > n) jobs[w].begin = n;
    if (jobs[w].end > n) jobs[w].end = n;
  }
  int rc = 0;
  if (nthreads == 1) {
    oracle_worker(&jobs[0]);
    rc = jobs[0].err ? 2 : 0;
  } else {
    int started = 0;
    for (int w = 0; w < nthreads; ++w) {
      if (pthread_create(&th[w], NULL, oracle_worker, &jobs[w]) != 0) { rc = 2; break; }
      ++started;
    }
    for (int w = 0; w < started; ++w) pthread_join(th[w], NULL);
    for (int w = 0; w < started; ++w) if (jobs[w].err) rc = 2;
  }
  free(jobs); free(th);
  return rc;
}
