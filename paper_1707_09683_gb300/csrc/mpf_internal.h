// mpf_internal.h -- structures shared by the host API and the scan kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mpf {

// Debug builds (compiled with -DMPF_DEBUG_CHECKS, libmpf_debug.so): kernels
// test their indexes against the buffers they were given; a failed test
// records kStatusBadIndex in the status word and the access is skipped, so
// nothing traps.  Release builds compile the tests away.
constexpr int kStatusBadIndex = 2;
#ifdef __CUDACC__
__device__ __forceinline__ void report_bad_index(int *status) {
  if (status) atomicCAS(status, 0, kStatusBadIndex);
}
// Dynamic shared memory of the running block, in bytes.
__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
  uint32_t r;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}
#endif
#ifdef MPF_DEBUG_CHECKS
#define MPF_DCHECK(status, cond) ((cond) || (mpf::report_bad_index(status), false))
#else
#define MPF_DCHECK(status, cond) true
#endif

// Residue code of padding rows.  Database sequences are padded with it to a
// 16-byte boundary; its table row scores kNegInf at every node, so a padding
// row leaves every score unchanged (the paper's '#' residue, Sec. 3.2).
constexpr int kPadCode = 32;
constexpr int kTableRows = 33;           // codes 0..31 plus padding
constexpr int kNegInf = -16384;          // score of padding rows and nodes > M
constexpr int kBlockThreads = 512;
constexpr int kMaxWords = 48;
constexpr int kStripedMaxM = 2 * 32 * kMaxWords;   // longest model of the striped kernels
constexpr int kMaxLongM = 100000;                  // longest model of the long-model kernel
constexpr int kLongThreads = 256;

enum Mode : int {
  MODE_SSV = 0,           // Alg. 7, 16-bit integer cells (DPX)
  MODE_MSV_FAST = 1,      // Alg. 2, begin score held constant between J changes
  MODE_MSV_DIRECT = 2,    // Alg. 2, J/B update after every row
  MODE_SSV_F16 = 3,       // MODE_SSV with cells as fp16 integers (FMA pipe)
  MODE_MSV_FAST_F16 = 4,  // MODE_MSV_FAST with cells as fp16 integers
  MODE_LONG_MSV = 5,      // models beyond kStripedMaxM, MSV: long_kernel
  MODE_TILE_SSV = 7,      // models beyond kStripedMaxM, SSV: tile_kernel<SSV>
  MODE_TILE_MSV = 8,      // models beyond kStripedMaxM, MSV when b may be held: tile_kernel<MSV>
                          //   (with MODE_LONG_MSV over the sequences it leaves)
  MODE_MSV_HELD = 9,      // Alg. 2 with the begin score held for the whole sequence: no per-row
                          //   tests; sequences whose running maximum passes T are listed and
                          //   rescored by MODE_MSV_DIRECT
  MODE_MSV_HELD_F16 = 10, // MODE_MSV_HELD with cells as fp16 integers
  MODE_MSV_SSV = 11,      // MODE_MSV_HELD and MODE_SSV from one sweep: with b held the MSV
                          //   cells minus b follow the SSV recurrence, so the largest cell
                          //   gives both filters' scores
  MODE_TILE_MSV_SSV = 12, // MODE_TILE_MSV and MODE_TILE_SSV from one sweep (the same reason)
};
constexpr int kNumModes = 8;   // modes of the striped scan kernel

// Striped kernels that read their table from tensor memory (one sequence per
// warp): the first tm_words(words) words of each lane's row of every residue
// code (all 33 rows: 33 x 14 = 462 of the 512 columns) come from TMEM, the
// rest from shared memory.
constexpr uint32_t kTmemColumns = 512;   // 32-bit columns of an SM's tensor memory
constexpr int kTmWordsAll = 14;     // lanes of up to this many words: all of them in TMEM
constexpr int kTmWordsPart = 12;    // longer lanes: this many in TMEM (a whole number of chunks)
constexpr int kTmMinWords = 8;      // fewer words per lane: the shared-memory kernels
// Words per lane read from TMEM for a lane of `words` words.  Twelve words
// take the shared-memory reads of a 48-word lane to 3/4 of the table, below
// the rate at which the integer pipe can use them.
__host__ __device__ constexpr int tm_words(int words) { return words <= kTmWordsAll ? words : kTmWordsPart; }

// Score-table formats: signed 16-bit integers, or the same integers as fp16.
// TABLE_I16_PACKED: integer scores in the packed geometry (one copy of each
// region; the tables of the queries that share a warp's sequence).
enum TableFormat : int { TABLE_I16 = 0, TABLE_F16 = 1, TABLE_I16_PACKED = 16 };
inline int table_format(int mode) {
  return (mode == MODE_SSV_F16 || mode == MODE_MSV_FAST_F16 || mode == MODE_MSV_HELD_F16) ? TABLE_F16
                                                                                           : TABLE_I16;
}

// One profile in one kernel layout (lives in device memory).
struct QueryDesc {
  const uint4 *table;     // shared-memory image: copies x 33 rows x quads x lanes
  uint32_t table_bytes;   // bytes to stage, multiple of 16 (includes smax)
  uint32_t row_bytes;     // stride between residue rows
  uint32_t copy_bytes;    // stride between bank-offset copies
  uint32_t smax_off;      // byte offset of 33 int16 per-code maximum scores
  uint32_t tail_off;      // byte offset of the two-word tail region (words % 4 == 2)
  uint32_t tail_row_bytes;
  int bias, tbm, tec, base, tjb_fixed;
  float scale;
  const uint8_t *tjb;     // per-length tjb (nullable)
  uint32_t n_tjb;
  uint32_t M;             // model length (long-model kernel)
  uint32_t seg_words;     // long-model kernel: cost words (4 nodes) per lane segment
  uint8_t *raw;           // outputs indexed by original sequence number
  uint8_t *flag;
  float *nat;             // nullable
  uint8_t *raw2;          // MODE_MSV_SSV: the SSV outputs (raw, flag above: MSV)
  uint8_t *flag2;
  float *nat2;            // nullable
  // Nullable: score only these length ranks (ascending), *n_ranks of them
  // (a device count written by an earlier kernel on the same stream).
  const uint32_t *ranks;
  const uint32_t *n_ranks;
  // Tiled MSV kernel and MSV_HELD: sequences left to an exact kernel (their
  // length ranks, and the count, zero before the launch).
  uint32_t *fallback_ranks;
  uint32_t *fallback_count;
};

struct ScanParams {
  const uint32_t *residues;   // residue words (4 codes each)
  uint32_t n_words;           // words in residues (debug index checks)
  const uint32_t *seq_word;   // per length rank: first word of the sequence
  const uint32_t *seq_len;    // per length rank: length
  const uint32_t *seq_orig;   // per length rank: original sequence number
  uint32_t n_seqs;
  uint32_t pad_word;          // a word of four padding codes
  const QueryDesc *queries;
  uint32_t n_queries;
  uint32_t n_shards;          // work item i = (query i / n_shards, shard i % n_shards)
  uint32_t *item_counter;     // zero before the launch
  int *status;                // nonzero: error reported by a kernel
  uint32_t long_words;        // long-model kernel: largest seg_words of its queries
  uint8_t *tile_col;          // tiled kernel: per resident warp two columns of
  uint32_t tile_col_stride;   //   tile_col_stride bytes (an int16 per row)
  uint64_t tile_col_bytes;
  uint32_t qp_table_stride;   // striped kernels with several queries per warp: bytes per staged table
};

typedef void (*KernelFn)(ScanParams);

// Long-model MSV kernel (mpf_long_kernel.cu, MODE_LONG_MSV), DP row as
// 16-bit pairs or (bytes) as bytes.
KernelFn long_kernel_for(int mode, bool bytes, int seg_words);
size_t long_smem_per_warp(int seg_words, bool bytes);

// Tiled kernel for long models (mpf_tile_kernel.cu, MODE_TILE_SSV and
// MODE_TILE_MSV): tiles of kTileNodes nodes, kTileC per lane, blocks of
// kTileWarps warps; per resident warp two columns of tile_col_stride bytes.
// Table: per tile [code 0..31][chunk 0..kTileC/8-1][lane] x 4 int16 pairs,
// pair p of lane l = nodes (l*kTileC + p, l*kTileC + p + kTileC/2), scores
// s = bias - cost (codes >= K: bias - 255; nodes past M: -32768); after the
// tiles (QueryDesc::smax_off) 32 int16 per-code maxima of s over the model.
constexpr int kTileC = 32;
constexpr int kTileNodes = 32 * kTileC;
constexpr int kTileWarps = 8;
constexpr int kTileWarpsTm = 16;
constexpr size_t kTileTableBytes = (size_t)32 * kTileNodes * 2;   // per tile
// The tiled kernel for a mode (MODE_TILE_*); tm: the tensor-memory variant
// (blocks of kTileWarpsTm warps, one per SM, the tile's scores in TMEM).
KernelFn tile_kernel_fn(int mode, bool tm);

// Stage-to-stage hand-off (mpf_pipeline.cu): SSV -> MSV (raw_bytes 1) and
// MSV -> Viterbi (raw_bytes 2).
constexpr int kSelectChunk = 4096;   // length ranks per selection block
int launch_select(const uint32_t *seq_orig, uint64_t n, int n_q, const uint8_t *in_flag,
                  const float *in_nat, float min_nat, void *out_raw, int raw_bytes,
                  uint8_t *out_flag, float *out_nat, uint32_t *chunk_count,
                  uint32_t *chunk_offset, uint32_t *ranks, uint32_t *n_ranks, cudaStream_t st);
int launch_pvalues(const float *nat, uint64_t n, float mu, float lambda, float *p, int num_sms,
                   cudaStream_t st);

// P7Viterbi filter (mpf_viterbi.cu).  Tables are int16 in device memory,
// striped (node l*Q + j in slot j*32 + l); -32768 is minus infinity.
constexpr int kVitFastMaxThreads = 512;
// Viterbi launch keys: kind * kVitKeyKind + the launch shape; queries with
// equal keys share a launch.
constexpr int kVitKeyKind = 1000000;
enum VitKind {
  kVitFastShared = 0,      // fast kernel, DP rows in shared memory
  kVitFastSharedNoD = 1,   // the same without the stored D row
  kVitGeneralShared = 2,   // general kernel, rows in shared memory
  kVitFastDevice = 3,      // fast kernel, rows in device memory (key + 1: without the stored D row)
  kVitGeneralDevice = 4,   // general kernel, rows in device memory
  kVitFastTeam = 5,        // fast kernel, a team of warps per sequence
  kVitFastDual = 6,        // both kinds 0/1 and 5, each taking the queries on its side of team_max
};
inline int vit_key_kind(int key) { return key / kVitKeyKind; }
inline bool vit_key_device_rows(int key) {
  return vit_key_kind(key) == kVitFastDevice || vit_key_kind(key) == kVitGeneralDevice;
}
constexpr int kVitRows = 32;         // msc rows: residue codes 0..31
constexpr int kVitTrans = 8;         // BM, MM, IM, DM, MI, II, MD, DD
constexpr int kVitSpecial = 8;       // NN, NB, EC, CC, CT, EJ, JJ, JB

// One query of a Viterbi launch (lives in device memory).
struct VitQuery {
  const int16_t *msc;         // kVitRows x Mpad match scores (codes >= K: -32768)
  const int16_t *trans;       // kVitTrans x Mpad
  int sp[kVitSpecial];
  int M, Mpad;                // nodes; row length, a multiple of 32
  int base;
  float scale;
  int16_t *score;             // outputs indexed by original sequence number
  uint8_t *flag;
  float *nat;                 // nullable
  const uint32_t *ranks;      // nullable: score only these length ranks (ascending),
  const uint32_t *n_ranks;    //   *n_ranks of them
  int64_t team_max;           // the team kernel scores the query when it selects at most
                              //   this many sequences, the one-warp kernels otherwise
};

struct VitParams {
  const uint32_t *residues;   // database words (4 codes each)
  uint32_t n_words;           // words in residues (debug index checks)
  int *status;                // debug index checks (nullable)
  const uint32_t *seq_word;   // per length rank
  const uint32_t *seq_len;
  const uint32_t *seq_orig;
  uint32_t n_seqs;
  uint32_t n_queries;
  int max_Mpad;               // largest Mpad of the queries (sets shared memory)
  const VitQuery *queries;
  uint32_t *counters;         // one per query, zero before the launch
  uint2 *state;               // models past the shared-memory rows: per-warp DP rows, else null
  uint64_t state_bytes;
};
// key: from viterbi_shape_key for the group's longest model (the kernel
// and launch shape; kinds with device rows need p.state).  Tables in the
// striped layout (msc [32][Q][32] int16, trans [Q][32] x 8 int16 with Q =
// Mpad / 32).  n_codes: distinct residue codes in the database (sizes the
// L1 share).  Returns 0, 1 on a CUDA error, 2 if the rows do not fit.
int launch_viterbi(const VitParams &p, int key, int n_codes, int max_smem, int num_sms, cudaStream_t st);
// Shared memory of a block of `warps` warps that store the D row.
size_t viterbi_fast_smem_bytes(int Mpad, int warps);
// Device scratch of a launch over models of up to Mpad nodes that keeps its
// rows in device memory.
size_t viterbi_state_bytes(bool fast, int Mpad, int num_sms);
// The VitQuery::team_max of a query with this key and length.
int64_t viterbi_team_max(int key, int Mpad, int n_codes, int max_smem, int num_sms);
// Launch key (kernel and launch shape) for one model length, or -1 if no
// shape fits.  fast: every transition and special score <= 0 (else the
// general kernel).  n_seqs: sequences each query of the launch scores, 0
// when the host does not know (a rank list counted on the device).
int viterbi_shape_key(bool fast, int Mpad, int n_codes, int max_smem, int num_sms, uint64_t n_seqs);

// Kernel instantiation for (lanes, words, mode), or nullptr if not built.
KernelFn kernel_for(int lanes, int words, int mode);
// The tensor-memory variant (lanes = 32), or nullptr if not built.
KernelFn kernel_lg32_tm(int words, int mode);
// Tensor-memory variants that score one sequence against 32 / lanes queries
// per warp (lanes 1 to 16), or nullptr if not built.
KernelFn kernel_qp_tm(int lanes, int words, int mode);
KernelFn kernel_qp_tm_lg1(int words, int mode);
KernelFn kernel_qp_tm_lg2(int words, int mode);
KernelFn kernel_qp_tm_lg4(int words, int mode);
KernelFn kernel_qp_tm_lg8(int words, int mode);
KernelFn kernel_qp_tm_lg16(int words, int mode);
KernelFn kernel_lg1(int words, int mode);
KernelFn kernel_lg2(int words, int mode);
KernelFn kernel_lg4(int words, int mode);
KernelFn kernel_lg8(int words, int mode);
KernelFn kernel_lg16(int words, int mode);
KernelFn kernel_lg32(int words, int mode);

// Shared-memory table geometry of a (lanes, words) layout.  Words 4q..4q+3
// of a lane are one 16-byte chunk of the quad region; when words % 4 == 2 the
// last two words of every lane are 8-byte chunks of a separate tail region.
//
// Quad region: for each residue row, the quads of the group's lanes are
// adjacent 16-byte chunks, so 8 lanes of one group (one phase of a 128-bit
// shared load) hit 8 distinct 16-byte bank groups.  Groups of fewer than 8
// lanes share a phase with other groups (other residues): the region then
// holds 8 / lanes copies with 128-byte aligned rows and bases offset by
// lanes * 16 bytes, and group g reads copy g mod copies.
// Tail region: a 64-bit load runs in phases of 16 lanes; each residue row is
// 128 bytes (256 for 32-lane groups) holding 16 / lanes copies of the
// group's 8-byte chunks side by side, and group g reads copy g mod copies.
// Packed geometry (the tables of queries that share a warp's sequence, each
// staged at its own offset): one copy of each region, tail rows of lanes x 8
// bytes.
struct TableGeom {
  int lanes, words, copies, quads, tail_words, tail_copies;
  uint32_t row_bytes, copy_bytes, tail_off, tail_row_bytes, smax_off, table_bytes;
};

inline TableGeom table_geom(int lanes, int words, bool packed = false) {
  TableGeom g;
  g.lanes = lanes;
  g.words = words;
  g.quads = words / 4;
  g.tail_words = words % 4;
  g.copies = (packed || lanes >= 8) ? 1 : 8 / lanes;
  uint32_t row = (uint32_t)g.quads * (uint32_t)lanes * 16u;
  if (g.copies > 1) row = (row + 127u) & ~127u;
  g.row_bytes = row;
  g.copy_bytes = (uint32_t)kTableRows * row + (g.copies > 1 ? (uint32_t)lanes * 16u : 0u);
  g.tail_off = (uint32_t)g.copies * g.copy_bytes;
  g.tail_off = (g.tail_off + 127u) & ~127u;
  g.tail_copies = (packed || lanes >= 16) ? 1 : 16 / lanes;
  g.tail_row_bytes = g.tail_words ? (uint32_t)(g.tail_copies * lanes * 8) : 0u;
  g.smax_off = g.tail_off + (uint32_t)kTableRows * g.tail_row_bytes;
  g.table_bytes = (g.smax_off + 80u + 15u) & ~15u;   // 33 int16, whole 16-byte chunks
  return g;
}

// Shared-memory bytes between the staged tables of a packed warp set
// (32 / lanes queries).  Rows of a phase's groups sit at the same table
// offset, so the stride spreads them over the banks: it is a multiple of
// 128 bytes plus lanes * 16 (at most 64; 0 for 16 lanes), which puts the
// 8 / lanes groups of a 128-bit phase on distinct 16-byte bank groups and
// the two 8-lane groups of a 64-bit tail phase on distinct halves.
inline uint32_t packed_table_stride(int lanes, int words) {
  const uint32_t tb = table_geom(lanes, words, true).table_bytes;
  const uint32_t off = lanes >= 16 ? 0u : (uint32_t)(lanes * 16 < 64 ? lanes * 16 : 64);
  return ((tb + 127u) & ~127u) + off;
}

}  // namespace mpf
