/*
 * mpf_vit_oracle.c -- scalar reference for the P7Viterbi filter.
 *
 * TEST INFRASTRUCTURE ONLY: the oracle the CUDA Viterbi kernel is checked
 * against.  Only the test suite and the CPU-baseline leg of the benchmark load
 * it.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (Eq. 1 of Sec. 2.1 with the Plan-7 special states, in the
 * 16-bit saturating word arithmetic of the HMMER3 Viterbi filter; insert
 * emissions score 0; local exits M_k -> E and D_k -> E score 0):
 *
 *   sat(v) = min(32767, max(-32768, v)); -32768 stands for minus infinity.
 *   row 0:  M[k] = I[k] = D[k] = -32768; xN = base; xB = sat(xN + tNB);
 *           xJ = xC = -32768
 *   for each residue x_i (previous-row values primed, M'[0] = I'[0] = D'[0] = -32768):
 *     M[k] = sat( max( sat(M'[k-1] + tMM[k]), sat(I'[k-1] + tIM[k]),
 *                      sat(D'[k-1] + tDM[k]), sat(xB + tBM[k]) ) + msc[x_i][k] )
 *     I[k] = max( sat(M'[k] + tMI[k]), sat(I'[k] + tII[k]) )      (k < M; I[M] = -32768)
 *     D[k] = max( sat(M[k-1] + tMD[k]), sat(D[k-1] + tDD[k]) )   (current row; D[1] = -32768)
 *     xE = max_k max(M[k], D[k]);  if xE == 32767 -> overflow
 *     xN = sat(xN + tNN); xC = max(sat(xC + tCC), sat(xE + tEC));
 *     xJ = max(sat(xJ + tJJ), sat(xE + tEJ)); xB = max(sat(xN + tNB), sat(xJ + tJB))
 *   score = sat(xC + tCT);  nat = (float)(score - base) / scale - 3 (or +inf on overflow)
 *
 * Residue codes >= K score -32768 as a match.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

enum { T_BM = 0, T_MM, T_IM, T_DM, T_MI, T_II, T_MD, T_DD, N_TRANS };
enum { X_NN = 0, X_NB, X_EC, X_CC, X_CT, X_EJ, X_JJ, X_JB, N_SPECIAL };

typedef struct {
  int M, K;
  const int16_t *msc;     /* K x M */
  const int16_t *trans;   /* N_TRANS x M, node k at index k-1 */
  const int16_t *special; /* N_SPECIAL */
  int base;
  float scale;
} vit_profile;

static int sat16(int v) { return v < -32768 ? -32768 : (v > 32767 ? 32767 : v); }
static int imax(int a, int b) { return a > b ? a : b; }

static int tr(const vit_profile *p, int t, int k) { return p->trans[(size_t)t * p->M + (k - 1)]; }

static void vit_one(const vit_profile *p, const uint8_t *seq, uint32_t L, int *Mr, int *Ir, int *Dr,
                    int *Mn, int *In, int *Dn, int16_t *score, uint8_t *flag, float *nat) {
  const int M = p->M;
  const int16_t *sp = p->special;
  for (int k = 0; k <= M; ++k) Mr[k] = Ir[k] = Dr[k] = -32768;
  int xN = p->base, xJ = -32768, xC = -32768;
  int xB = sat16(xN + sp[X_NB]);
  for (uint32_t i = 0; i < L; ++i) {
    const int x = seq[i];
    Mn[0] = In[0] = Dn[0] = -32768;
    int xE = -32768;
    for (int k = 1; k <= M; ++k) {
      int best = sat16(Mr[k - 1] + tr(p, T_MM, k));
      best = imax(best, sat16(Ir[k - 1] + tr(p, T_IM, k)));
      best = imax(best, sat16(Dr[k - 1] + tr(p, T_DM, k)));
      best = imax(best, sat16(xB + tr(p, T_BM, k)));
      const int e = x < p->K ? p->msc[(size_t)x * M + (k - 1)] : -32768;
      Mn[k] = sat16(best + e);
      In[k] = k < M ? imax(sat16(Mr[k] + tr(p, T_MI, k)), sat16(Ir[k] + tr(p, T_II, k))) : -32768;
      Dn[k] = k > 1 ? imax(sat16(Mn[k - 1] + tr(p, T_MD, k)), sat16(Dn[k - 1] + tr(p, T_DD, k))) : -32768;
      xE = imax(xE, imax(Mn[k], Dn[k]));
    }
    if (xE >= 32767) {
      *score = 32767; *flag = 1; *nat = INFINITY;
      return;
    }
    xN = sat16(xN + sp[X_NN]);
    xC = imax(sat16(xC + sp[X_CC]), sat16(xE + sp[X_EC]));
    xJ = imax(sat16(xJ + sp[X_JJ]), sat16(xE + sp[X_EJ]));
    xB = imax(sat16(xN + sp[X_NB]), sat16(xJ + sp[X_JB]));
    int *t;
    t = Mr; Mr = Mn; Mn = t;
    t = Ir; Ir = In; In = t;
    t = Dr; Dr = Dn; Dn = t;
  }
  const int sc = sat16(xC + sp[X_CT]);
  *score = (int16_t)sc;
  *flag = 0;
  *nat = (float)(sc - p->base) / p->scale - 3.0f;
}

typedef struct {
  const vit_profile *p;
  const uint8_t *residues;
  const uint64_t *offsets;
  const uint32_t *lengths;
  const uint64_t *index;
  int16_t *score;
  uint8_t *flag;
  float *nat;
  uint64_t begin, end;
  int err;
} vit_job;

static void *vit_worker(void *arg) {
  vit_job *j = (vit_job *)arg;
  const size_t m1 = (size_t)j->p->M + 1;
  int *buf = (int *)malloc(sizeof(int) * m1 * 6);
  if (!buf) { j->err = 1; return NULL; }
  for (uint64_t q = j->begin; q < j->end; ++q) {
    const uint64_t s = j->index ? j->index[q] : q;
    vit_one(j->p, j->residues + j->offsets[s], j->lengths[s], buf, buf + m1, buf + 2 * m1,
            buf + 3 * m1, buf + 4 * m1, buf + 5 * m1, &j->score[q], &j->flag[q], &j->nat[q]);
  }
  free(buf);
  return NULL;
}

/*
 * Score sequences with the Viterbi filter.  Host pointers.
 *   msc: K x M int16; trans: 8 x M int16 in the order BM, MM, IM, DM, MI, II,
 *   MD, DD (node k at index k-1); special: 8 int16 NN, NB, EC, CC, CT, EJ, JJ, JB.
 * Returns 0, 1 on bad arguments, 2 on allocation failure.
 */
int oracle_viterbi(int M, int K, const int16_t *msc, const int16_t *trans, const int16_t *special,
                   int base, float scale, const uint8_t *residues, const uint64_t *offsets,
                   const uint32_t *lengths, const uint64_t *index, uint64_t n, int16_t *score,
                   uint8_t *flag, float *nat, int nthreads) {
  if (M < 1 || K < 1 || K > 32 || !msc || !trans || !special) return 1;
  if (n > 0 && (!residues || !offsets || !lengths || !score || !flag || !nat)) return 1;
  vit_profile p = {M, K, msc, trans, special, base, scale};
  if (nthreads < 1) nthreads = 1;
  if ((uint64_t)nthreads > n) nthreads = n > 0 ? (int)n : 1;
  vit_job *jobs = (vit_job *)calloc((size_t)nthreads, sizeof(vit_job));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return 2; }
  const uint64_t chunk = (n + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
  for (int w = 0; w < nthreads; ++w) {
    uint64_t b = (uint64_t)w * chunk, e = b + chunk;
    if (b > n) b = n;
    if (e > n) e = n;
    jobs[w] = (vit_job){&p, residues, offsets, lengths, index, score, flag, nat, b, e, 0};
  }
  int rc = 0, started = 0;
  for (int w = 0; w < nthreads; ++w) {
    if (nthreads == 1) { vit_worker(&jobs[0]); break; }
    if (pthread_create(&th[w], NULL, vit_worker, &jobs[w]) != 0) { rc = 2; break; }
    ++started;
  }
  for (int w = 0; w < started; ++w) pthread_join(th[w], NULL);
  for (int w = 0; w < nthreads; ++w) if (jobs[w].err) rc = 2;
  free(jobs); free(th);
  return rc;
}
