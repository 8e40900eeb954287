/*
 * mpf.h -- C ABI of the GB300 MSV/SSV protein-profile scan library (libmpf.so).
 *          (The P7Viterbi filter that follows them is declared further down.)
 *
 * The library scores every sequence of a protein database against Plan-7
 * profiles with the two byte-quantised heuristic filters of the HMMER3
 * pipeline (Sec. 2.1 of CUDAMPF++, arXiv 1707.09683):
 *
 *   MSV  -- ungapped local alignment with multiple hits: Insert and Delete
 *           states pruned, the M->M transition scored 0, hits chained through
 *           the J state.  Byte update of Alg. 2:
 *             dp[k] = sat(sat(max(dp'[k-1], xB) + bias) - cost[x][k])
 *             xE = max_k dp[k];  overflow when xE >= 255 - bias
 *             xJ = max(xJ, sat(xE - tec));  xB = sat(max(base, xJ) - (tjb + tbm))
 *           raw score = xJ, nat = (raw - tjb - base) / scale - 3.
 *   SSV  -- the MSV model with the J state removed (single segment), Alg. 7,
 *           read in unsigned offset form:
 *             r[k] = min(255, max(0, r'[k-1] + bias - cost[x][k])),  R = max r
 *           overflow when R == 255; nat = (R - tbm - tec - 2 tjb) / scale - 3.
 *   sat(v) = min(255, max(0, v)); dp', r' are the previous row; xB starts at
 *   sat(base - (tjb + tbm)), xJ at 0, dp and r at 0.
 *
 * Per sequence the library returns the raw byte score, an exact overflow
 * (saturation) flag and the nat score.  Overflow is not an error: its raw
 * score is 255 and its nat score +inf.  Results are bit-identical to the
 * scalar definition above for every input.
 *
 * Conventions (all entry points):
 *   - Return 0 (MPF_OK) or a positive MPF_E* code; never abort.  After
 *     MPF_ECUDA the context should be destroyed.
 *   - Inputs are copied; the caller keeps ownership of its buffers.  Handles
 *     are owned by the caller and released with the matching *_destroy, which
 *     accepts NULL.  A profile or database may be used with any context on
 *     the device it was created on (contexts are streams: several contexts
 *     can scan one resident database concurrently); it must be destroyed
 *     before the context it was created in, and only after the scans that
 *     use it have completed (scans queued on its own context's stream are
 *     ordered before the release automatically).
 *   - Output buffers are caller-allocated and may be host or device memory
 *     (detected per pointer).  With device outputs a scan is asynchronous on
 *     the context stream; call mpf_sync() (or synchronise that stream) before
 *     reading them.  With host outputs the call copies back and returns when
 *     the results are in place.
 *   - One context may be used by one host thread at a time.
 */
#ifndef MPF_H
#define MPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpf_ctx mpf_ctx;
typedef struct mpf_profile mpf_profile;
typedef struct mpf_db mpf_db;

enum {
  MPF_OK = 0,
  MPF_EINVAL = 1,       /* bad argument (null handle, size out of range, code >= 32 ...) */
  MPF_ENOMEM = 2,       /* host or device allocation failed                              */
  MPF_ECUDA = 3,        /* a CUDA runtime call failed                                    */
  MPF_ETIMEOUT = 4,     /* a bounded device wait gave up (status word set by a kernel)    */
  MPF_EUNSUPPORTED = 5, /* valid request the library does not handle (e.g. M too large)  */
  MPF_EDEVICE = 6       /* a kernel's index check failed (only libmpf_debug.so checks)    */
};

/* Filters.  MPF_MSV_SSV (batches and plans only) asks for both: see
 * mpf_scan_batch. */
enum { MPF_MSV = 0, MPF_SSV = 1, MPF_MSV_SSV = 2 };

/* Largest model length M a byte-filter or Viterbi profile may have (100,000). */
int mpf_max_model_length(void);

/* Largest model length the striped shared-memory scan kernels hold (3,072).
 * Longer byte-filter profiles are scored by the long-model kernels, one
 * warp per sequence: the model swept in tiles of 1,024 nodes with the DP
 * row in registers (SSV; MSV with the begin score held, rescoring exactly
 * the sequences where it would move), or each lane a contiguous segment of
 * nodes with the row in shared memory (MSV otherwise).  The paper's tables
 * end at M = 2405; models beyond the on-chip table are the large-model case
 * of its Sec. 6.  Longer Viterbi profiles keep their DP rows in device
 * memory instead of shared memory. */
int mpf_max_striped_length(void);

/* Message for a status code (static string, never NULL). */
const char *mpf_strerror(int status);

/*
 * Create a context on CUDA device `device`.
 *   cuda_stream: a cudaStream_t created by the caller on that device (kept,
 *                not owned), or NULL for a library-owned non-blocking stream.
 * Errors: MPF_EINVAL (bad device or out == NULL), MPF_ECUDA, MPF_ENOMEM.
 */
int mpf_ctx_create(int device, void *cuda_stream, mpf_ctx **out);
void mpf_ctx_destroy(mpf_ctx *ctx);

/* The cudaStream_t the context launches on (for events and interop). */
void *mpf_ctx_stream(mpf_ctx *ctx);

/* Wait for all work queued on the context stream.  Returns MPF_EDEVICE if a
 * kernel of the debug build (libmpf_debug.so) found an index outside the
 * buffers it was given (the access was skipped, results are not valid), and
 * reserves MPF_ETIMEOUT for a bounded device wait that gave up (the current
 * kernels have no device-side waits).  The status stays set until the
 * context is destroyed. */
int mpf_sync(mpf_ctx *ctx);

/*
 * Create a profile from biased match costs (the emission-score table E of
 * Alg. 2 / Alg. 4, here as cost bytes; the paper extends the alphabet to 32
 * codes, Sec. 3.3).
 *   M:      model length, 1 <= M <= mpf_max_model_length()
 *   K:      residue codes with costs, 1 <= K <= 32; codes K..31 cost 255
 *   cost:   host pointer, K*M bytes, row-major [x][k-1] (node k of residue x)
 *   bias_b, tbm_b, tec_b, base_b: the bias, B->M entry, E->C/J exit and
 *           base bytes of the recurrences above
 *   tjb_b:  the N/C/J loop byte used when tjb_by_len is NULL
 *   tjb_by_len: nullable host pointer of n_tjb bytes: tjb for sequence length
 *           L is tjb_by_len[min(L, n_tjb - 1)] (Alg. 2 derives the begin score
 *           of each sequence from its length)
 *   scale_b: units per nat of the nat score (finite, > 0)
 * The profile keeps copies of cost and tjb_by_len.  Results are the same
 * exact recurrences whichever kernel runs (striped up to
 * mpf_max_striped_length(), long-model above).
 * Errors: MPF_EINVAL, MPF_EUNSUPPORTED (M too large), MPF_ENOMEM, MPF_ECUDA.
 */
int mpf_profile_create(mpf_ctx *ctx, int M, int K, const uint8_t *cost, uint8_t bias_b,
                       uint8_t tbm_b, uint8_t tec_b, uint8_t tjb_b, const uint8_t *tjb_by_len,
                       uint32_t n_tjb, float scale_b, uint8_t base_b, mpf_profile **out);
void mpf_profile_destroy(mpf_profile *prof);

/*
 * Kernel configuration of a profile for one filter: `lanes` threads of a warp
 * share one sequence (1, 2, 4, 8, 16 or 32) and each holds `words` 32-bit
 * words of two 16-bit cells (4 <= words <= 48, even), so the striped
 * model holds 2 * lanes * words >= M cells (Sec. 3.1: S = 32 / lanes
 * sequences per warp, W = 2 * lanes cells per row step, H = words).
 * set: MPF_EINVAL if the pair is not built or does not cover M, or if the
 *      profile is longer than mpf_max_striped_length() (one configuration).
 * get: writes the pair the next scan will use (tuned default if never set);
 *      lanes 32, words 0 for the long-model kernel.
 */
int mpf_profile_set_config(mpf_profile *prof, int filter, int lanes, int words);
int mpf_profile_get_config(const mpf_profile *prof, int filter, int *lanes, int *words);

/*
 * On-chip and device-memory footprint of a profile's scans with one filter
 * (for admission control by a server; not in the paper).  smem_bytes: the
 * shared memory one thread block of its kernel takes (the staged score table
 * or tile; for the lane-segment long-model kernel, one warp's DP row), with
 * the configuration the next scan will use.  table_bytes: the device memory
 * the profile's score tables for that kernel hold once built.  A scan also
 * writes 6 bytes per database sequence (raw, flag, nat) into the caller's
 * buffers.
 * Errors: MPF_EINVAL (null pointer or bad filter).
 */
int mpf_profile_footprint(const mpf_profile *prof, int filter, uint32_t *smem_bytes,
                          uint64_t *table_bytes);

/*
 * Cell arithmetic of a profile's scans for one filter.  Both give identical
 * results (the recurrences stay exact): MPF_ARITH_I16 updates two 16-bit
 * integer cells per DPX instruction on the integer pipe, MPF_ARITH_F16 holds
 * the same integers as half-precision values and updates them with a fused
 * add-and-clamp on the FMA pipe.  MPF_ARITH_AUTO (default) is MPF_ARITH_I16:
 * no floating point in the cell updates.
 * Errors: MPF_EINVAL.
 */
enum { MPF_ARITH_AUTO = 0, MPF_ARITH_I16 = 1, MPF_ARITH_F16 = 2 };
int mpf_profile_set_arith(mpf_profile *prof, int filter, int arith);

/*
 * Where a scan reads its score table (not in the paper, whose Alg. 4 reads
 * it through the read-only cache).  Every striped kernel stages the table in
 * shared memory; with one sequence per warp (lanes 32, words >= 8) the
 * automatic choice also copies the first words of each lane's row (all of
 * them up to 14 words per lane, else 12) into the SM's tensor memory (TMEM,
 * read by tcgen05.ld at about three times the shared-memory rate) and reads
 * those words from there.  For long models the tiled kernels' automatic
 * choice holds each 1,024-node tile in TMEM instead of shared memory (one
 * block of 16 warps per SM).  Results are identical either way.
 *   set: MPF_TABLE_AUTO (default) or MPF_TABLE_SHARED (shared memory only).
 *   get: MPF_TABLE_TENSOR or MPF_TABLE_SHARED, for the configuration the
 *        next scan will use.
 * Errors: MPF_EINVAL.
 */
enum { MPF_TABLE_AUTO = 0, MPF_TABLE_SHARED = 1, MPF_TABLE_TENSOR = 2 };

/*
 * Work decomposition of a profile's striped scans with one filter (replaces
 * the static thread-block assignment of Sec. 3.1 and the warp data blocks of
 * Alg. 1): the database's length ranks are dealt round-robin into
 * factor x (resident blocks) shards, and blocks pull (query, shard) work
 * items.  More shards make smaller items, so blocks finish closer together,
 * at the cost of staging the table once per item.  1 <= factor <= 16
 * (default 1); a launch takes the largest factor of its queries; long models
 * ignore it.  Results do not depend on it.
 * Errors: MPF_EINVAL.
 */
int mpf_profile_set_shard_factor(mpf_profile *prof, int filter, int factor);
int mpf_profile_get_shard_factor(const mpf_profile *prof, int filter, int *factor);
int mpf_profile_set_table_memory(mpf_profile *prof, int filter, int where);
int mpf_profile_get_table_memory(const mpf_profile *prof, int filter, int *where);

/*
 * Upload a database of digital sequences (host pointers).
 *   residues: n_residues codes, each < 32
 *   offsets, lengths: n_seqs entries; sequence s is
 *             residues[offsets[s] .. offsets[s] + lengths[s]); lengths may be 0
 * The database is copied into device memory (length-sorted, 16-byte aligned
 * sequences; Sec. 3.2 replaced by a sorted layout) and stays resident.
 * Errors: MPF_EINVAL (code >= 32, range outside residues, n_seqs >= 2^31),
 *         MPF_ENOMEM, MPF_ECUDA.
 */
int mpf_db_upload(mpf_ctx *ctx, const uint8_t *residues, uint64_t n_residues,
                  const uint64_t *offsets, const uint32_t *lengths, uint64_t n_seqs,
                  mpf_db **out);
void mpf_db_destroy(mpf_db *db);
uint64_t mpf_db_n_seqs(const mpf_db *db);
uint64_t mpf_db_n_residues(const mpf_db *db);

/*
 * Score every database sequence with one profile (one kernel launch).
 *   raw, overflow: n_seqs bytes each; nat: n_seqs floats or NULL.
 *   Output index = sequence number in the uploaded order.
 * Errors: MPF_EINVAL, MPF_ENOMEM, MPF_ECUDA, MPF_ETIMEOUT (host outputs).
 */
int mpf_msv_scan(mpf_ctx *ctx, const mpf_profile *prof, const mpf_db *db, uint8_t *raw,
                 uint8_t *overflow, float *nat);
int mpf_ssv_scan(mpf_ctx *ctx, const mpf_profile *prof, const mpf_db *db, uint8_t *raw,
                 uint8_t *overflow, float *nat);

/*
 * Score the database with n_q profiles in one persistent launch per kernel
 * configuration (work items of (query, database shard) pulled by resident
 * thread blocks; launches of different configurations overlap).
 *   filter: MPF_MSV, MPF_SSV or MPF_MSV_SSV
 *   raw, overflow: n_q * n_seqs bytes, nat: n_q * n_seqs floats or NULL,
 *   query-major ([q][s]).  MPF_MSV_SSV: twice that, the MSV block ([q][s])
 *   then the SSV block.
 * Results equal n_q separate mpf_msv_scan / mpf_ssv_scan calls.
 * MPF_MSV_SSV scores a query once for both filters where it can: with the
 * begin score held (the MSV pass used when the first begin score of every
 * sequence is below 255 - bias, Alg. 2), the MSV cells less the begin score
 * follow the SSV recurrence (Alg. 7), so one sweep's largest cell gives both
 * scores.  That needs integer cells for both filters and the same
 * configuration and table memory for both (mpf_profile_set_config,
 * mpf_profile_set_table_memory; the MSV shard factor is used); long models
 * whose MSV runs the held tiled pass sweep their tiles once for both.  Other
 * queries run each filter's kernels.
 * Errors: as the single scans.
 */
int mpf_scan_batch(mpf_ctx *ctx, int filter, const mpf_profile *const *profs, int n_q,
                   const mpf_db *db, uint8_t *raw, uint8_t *overflow, float *nat);

/*
 * Reusable launch plans (device outputs only).  A plan fixes the profiles,
 * the database and the output buffers of a batch; launching it enqueues the
 * scan on the context stream without host synchronisation or allocation.
 * Queries whose kernel configurations differ run as separate kernels that
 * overlap (forked streams, joined back into the context stream).  In a plan
 * of two or more queries, those with fewer than 32 lanes per sequence
 * (integer SSV, held MSV or both, table memory not set to MPF_TABLE_SHARED,
 * at least 8 words) may be packed 32 / lanes to a warp: the warp scores one
 * sequence against all of them, with the score rows in tensor memory.
 * Packed queries are sorted by words per lane; runs of them form sets where
 * a cost model in warp-words per row says a set pays, and each takes the
 * largest word count of its set (the added nodes score as padding: the
 * outputs do not change).
 *   mpf_plan_create:  arguments as mpf_scan_batch; raw/overflow/nat must be
 *                     device pointers (MPF_EINVAL otherwise).  The plan keeps
 *                     pointers to the profiles and database: they must outlive it.
 *   mpf_plan_launch:  enqueue one run (asynchronous).
 *   mpf_plan_capture_graph: record the run as a CUDA graph; later launches
 *                     replay the graph.  Call it outside any stream capture.
 *   mpf_plan_kernel_launches: scan kernels one run launches (>= 1), the
 *                     exact-rescoring launches after held or tiled MSV passes
 *                     included.
 *   mpf_plan_group_count: launch groups of the plan (the kernels of one run
 *                     before any rescoring launch); 0 for a NULL plan.
 *   mpf_plan_group_info: group i's kernel configuration: lanes per sequence,
 *                     words per lane (0: tiled or long-model kernel), where
 *                     its table is read from (MPF_TABLE_SHARED or
 *                     MPF_TABLE_TENSOR), queries scored per warp and
 *                     sequence (1, or 32 / lanes when packed), its number
 *                     of queries and the filters it scores (1: MSV, 2: SSV,
 *                     3: both in one sweep).  Any output pointer may be NULL;
 *                     MPF_EINVAL for a NULL plan or i out of range.
 *   mpf_plan_pack_sets: the packed sets a plan forms among n queries of
 *                     `lanes` lanes per sequence (1, 2, 4, 8 or 16) with
 *                     these words per lane (ascending), blocks having
 *                     max_smem bytes of shared memory: set_start[i] is the
 *                     index of the first query of query i's set, or -1 when
 *                     query i keeps its one-query kernel.  The sets are runs
 *                     of at most 32 / lanes queries that minimise a cost in
 *                     warp-words per row: (32 / lanes) x the set's largest
 *                     words for a set, 5/4 of its own words for a query
 *                     alone.  Host only.  MPF_EINVAL for other lanes, n < 0,
 *                     NULL arrays, or words not ascending or below 1.
 *   mpf_plan_destroy: waits for the context stream, then frees the plan.
 */
typedef struct mpf_plan mpf_plan;
int mpf_plan_create(mpf_ctx *ctx, int filter, const mpf_profile *const *profs, int n_q,
                    const mpf_db *db, uint8_t *raw, uint8_t *overflow, float *nat,
                    mpf_plan **out);
int mpf_plan_launch(mpf_plan *plan);
int mpf_plan_capture_graph(mpf_plan *plan);
int mpf_plan_kernel_launches(const mpf_plan *plan);
int mpf_plan_group_count(const mpf_plan *plan);
int mpf_plan_pack_sets(int lanes, const int *words, int n, int max_smem, int *set_start);
int mpf_plan_group_info(const mpf_plan *plan, int i, int *lanes, int *words, int *table_memory,
                        int *queries_per_warp, int *n_queries, int *filters);
void mpf_plan_destroy(mpf_plan *plan);

/*
 * Two-stage filter of the HMMER3 pipeline (Sec. 2.1): SSV scores every
 * sequence; the sequences whose SSV nat score is >= ssv_min_nat, or whose SSV
 * score overflowed, are re-scored by MSV; the others are marked filtered.
 *   All buffers are device pointers; outputs [n_q][n_seqs] by original
 *   sequence number.  ssv_* receive the SSV scores of every sequence; msv_*
 *   receive the MSV scores of the passing sequences and raw 0, flag 2, nat NaN
 *   for filtered ones (msv_nat nullable).  n_pass[n_q] receives the number of
 *   passing sequences per query.
 *   Asynchronous on the context stream (one SSV and one MSV launch per kernel
 *   configuration, three selection kernels between them); temporary device
 *   memory is taken from and returned to the stream-ordered pool.
 * The seven buffers must not overlap one another: the hand-off reads the SSV
 * outputs while it writes the MSV ones.
 * Errors: MPF_EINVAL (null or host buffer, NaN threshold, overlapping
 * buffers), MPF_ENOMEM, MPF_ECUDA.
 */
int mpf_pipeline_scan(mpf_ctx *ctx, const mpf_profile *const *profs, int n_q, const mpf_db *db,
                      float ssv_min_nat, uint8_t *ssv_raw, uint8_t *ssv_flag, float *ssv_nat,
                      uint8_t *msv_raw, uint8_t *msv_flag, float *msv_nat, uint32_t *n_pass);

/*
 * P-values of nat scores under a Gumbel (extreme-value) distribution with
 * location mu and slope lambda > 0: P(S > x) = 1 - exp(-exp(-lambda (x - mu)))
 * (the per-sequence P-value of Alg. 2 and Alg. 7; mu and lambda come from
 * the caller's calibration).  +inf (overflow) gives 0, NaN (filtered) stays
 * NaN.  nat and p are device pointers of n floats (may alias); single
 * precision; asynchronous on the context stream.
 * Errors: MPF_EINVAL, MPF_ECUDA.
 */
int mpf_pvalues(mpf_ctx *ctx, const float *nat, uint64_t n, float mu, float lambda, float *p);

/*
 * P7Viterbi filter: the gapped Viterbi recurrence of Eq. 1 (Sec. 2.1), the
 * third filter of the HMMER3 pipeline, in 16-bit saturating word arithmetic:
 *
 *   sat(v) = min(32767, max(-32768, v)); -32768 stands for minus infinity;
 *   primed values are the previous row; M'[0] = I'[0] = D'[0] = -32768.
 *   row 0:  M = I = D = -32768; xN = base; xB = sat(xN + NB); xJ = xC = -32768
 *   residue x:
 *     M[k] = sat(max(sat(M'[k-1] + MM[k]), sat(I'[k-1] + IM[k]),
 *                    sat(D'[k-1] + DM[k]), sat(xB + BM[k])) + msc[x][k])
 *     I[k] = max(sat(M'[k] + MI[k]), sat(I'[k] + II[k]))   for k < M; I[M] = -32768
 *     D[k] = max(sat(M[k-1] + MD[k]), sat(D[k-1] + DD[k])) for k > 1; D[1] = -32768
 *     xE = max over k of max(M[k], D[k]); xE >= 32767 -> overflow (stop)
 *     xN = sat(xN + NN);  xC = max(sat(xC + CC), sat(xE + EC));
 *     xJ = max(sat(xJ + JJ), sat(xE + EJ));  xB = max(sat(xN + NB), sat(xJ + JB))
 *   score = sat(xC + CT); nat = (score - base) / scale - 3 (float; +inf on overflow)
 *
 * Insert states emit with score 0 and every match and delete state may exit
 * to E with score 0 (local alignment).
 */
typedef struct mpf_vprofile mpf_vprofile;

/*
 * Create a Viterbi profile.  Host inputs, copied.
 *   M: 1 <= M <= mpf_max_model_length(); K: 1 <= K <= 32 residue codes
 *   msc: K*M int16, row-major [x][k-1] match scores; codes K..31 score -32768
 *   trans: 8*M int16, rows BM, MM, IM, DM, MI, II, MD, DD, column k-1 holds
 *          the transition into (BM, MM, IM, DM: M_k; MD, DD: D_k) or out of
 *          (MI, II: I_k) node k
 *   special: 8 int16 NN, NB, EC, CC, CT, EJ, JJ, JB
 *   base: the score offset, -32768..32767; scale: units per nat (finite, > 0)
 * Errors: MPF_EINVAL, MPF_EUNSUPPORTED (M too large), MPF_ENOMEM, MPF_ECUDA.
 */
int mpf_vit_profile_create(mpf_ctx *ctx, int M, int K, const int16_t *msc, const int16_t *trans,
                           const int16_t *special, int base, float scale, mpf_vprofile **out);
/* Waits for the creating context's stream, then frees the profile. */
void mpf_vit_profile_destroy(mpf_vprofile *vprof);

/*
 * Score every database sequence against n_q Viterbi profiles.
 *   score [n_q][n_seqs] int16, overflow [n_q][n_seqs] bytes (0 or 1), nat
 *   [n_q][n_seqs] floats or NULL, by original sequence number; host or device
 *   buffers, as for the byte scans (one kernel launch for all queries).
 * Errors: MPF_EINVAL, MPF_EUNSUPPORTED, MPF_ENOMEM, MPF_ECUDA.
 */
int mpf_viterbi_scan(mpf_ctx *ctx, const mpf_vprofile *const *vprofs, int n_q, const mpf_db *db,
                     int16_t *score, uint8_t *overflow, float *nat);

/*
 * Third stage of the pipeline (Sec. 2.1): re-score with the Viterbi filter
 * the sequences that passed MSV.  msv_flag / msv_nat are the MSV outputs of
 * mpf_pipeline_scan (or of an MSV scan), [n_q][n_seqs] device buffers; a
 * sequence passes when its MSV flag is 1 (overflow) or its MSV nat score is
 * >= msv_min_nat (flag 2, filtered by SSV, never passes).  Passing sequences
 * receive their Viterbi score, flag and nat; the others score -32768, flag 2,
 * nat NaN.  n_pass[n_q] receives the number of passing sequences per query.
 * All buffers are device pointers (nat nullable); asynchronous on the context
 * stream; temporary device memory comes from the stream-ordered pool.  The
 * buffers must not overlap one another (the MSV inputs are read while the
 * Viterbi outputs are written).
 * Errors: MPF_EINVAL (null or host buffer, NaN threshold, overlapping
 * buffers), MPF_EUNSUPPORTED, MPF_ENOMEM, MPF_ECUDA.
 */
int mpf_viterbi_rescore(mpf_ctx *ctx, const mpf_vprofile *const *vprofs, int n_q, const mpf_db *db,
                        const uint8_t *msv_flag, const float *msv_nat, float msv_min_nat,
                        int16_t *score, uint8_t *overflow, float *nat, uint32_t *n_pass);

/*
 * Self-test of the kernels' debug index checks (libmpf_debug.so only: the
 * library built with -DMPF_DEBUG_CHECKS, whose kernels test every index they
 * derive from their inputs against the buffers they were given, skip the
 * access and record the failure in the context's status word).  Launches one
 * block whose check fails with no access behind it; the next mpf_sync on the
 * context returns MPF_EDEVICE, as do all later ones (the status is sticky:
 * use a context of its own).  The paper has no counterpart: this stands in
 * for a memory checker on a pool where none is available.
 * Errors: MPF_EINVAL (null context), MPF_EUNSUPPORTED (release library),
 * MPF_ECUDA.
 */
int mpf_debug_check_selftest(mpf_ctx *ctx);

/*
 * Allocation-free scan.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory when they score, such as
 * services that account for all device memory up front and run under a fixed
 * budget, or plug-ins whose host application owns the device allocator (its
 * pool holds the memory, and a cudaMalloc beside it can fail or stall the
 * device).  It scores like mpf_msv_scan / mpf_ssv_scan (filter = MPF_MSV or
 * MPF_SSV) but calls no cudaMalloc, cudaFree or other allocating routine: its
 * query descriptor, work counter and striped cost table live in one
 * file-scope device array of 512 + 224 KiB = 229,888 bytes that every GPU
 * loading the library holds until the process exits.  The kernel reports
 * through the context's status word, as the regular scans do.
 *   raw, overflow: device pointers, n_seqs bytes each; nat: device pointer of
 *     n_seqs floats or NULL.  Host pointers are rejected (MPF_EINVAL).
 *   Asynchronous on the context stream, like a scan into device outputs.
 *   A profile whose table image for the chosen kernel configuration exceeds
 *     224 KiB is rejected with MPF_EUNSUPPORTED (none of the built
 *     configurations does; the largest needs 202,832 bytes), and so is a
 *     profile longer than mpf_max_striped_length().
 *   The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any
 *     stream capture.
 *   All calls share the one array and each call overwrites it (the counter
 *     is cleared on the stream): calls ordered on one stream
 *     are safe, calls whose kernels overlap on the GPU (other streams or
 *     contexts on the same device) race and give wrong results.
 * Errors: MPF_EINVAL, MPF_EUNSUPPORTED, MPF_ECUDA.
 */
int mpf_scan_noalloc(mpf_ctx *ctx, int filter, const mpf_profile *prof, const mpf_db *db,
                     uint8_t *raw, uint8_t *overflow, float *nat);

#ifdef __cplusplus
}
#endif

#endif /* MPF_H */
