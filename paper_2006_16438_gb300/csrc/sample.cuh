// SkrpLev (Alg. 1) on the GPU: deterministic rows (Section 5.3), random rows with
// rejection (Alg. 2), CombineRepeats (Section 4.1) -- all without host round trips.
#pragma once

#include "dense.cuh"

namespace cpa {

constexpr int kXsLimbs = 36;  // exact-sum accumulator: 36 x 32 bits from 2^-1074 up
constexpr int kXsRep = 8;     // replicas of the accumulator (blocks spread their atomics)

// Device scalars of one sampling pass.
struct SampleState {
  int status;
  int no_det;
  int need_topk;
  int pad0;
  int64_t ncand[kMaxOrder];
  uint64_t cand_total;
  uint64_t det_count;   // rows that passed p_i > tau (may exceed s)
  int64_t sdet;
  int64_t srnd;
  int64_t nsort;        // sdet + srnd
  int64_t sbar;         // rows after combining
  int64_t nuniq;        // distinct keys in the sorted buffer
  uint64_t attempts;
  uint64_t slot_ctr;    // next random slot to hand out (work queue of the draws)
  double pdet;
  double alpha_star;
  double thr[kMaxOrder];
  uint64_t xs[kXsRep * kXsLimbs];  // exact-sum bins of p_det; the sum is over the replicas
};

// Per-mode distributions of the d other modes (device pointers): the inclusive
// fixed-point CDF, its summary, and p_t(i) = q_i / T_t precomputed per row.
struct OtherDists {
  const uint64_t* C[kMaxOrder];
  const DistInfo* info[kMaxOrder];
  const double* P[kMaxOrder];
};

// p[i] = q_i / T (q_i = C_i - C_{i-1}), the IEEE quotient the sampler uses.
int phat_from_cdf(const uint64_t* C, int64_t n, const DistInfo* info, double* p, cudaStream_t st);

struct SampleParams {
  KeyLayout L;          // other modes of the update
  OtherDists D;
  int64_t s;
  double tau;
  uint64_t seed;
  uint64_t iter;               // outer iteration of the Philox counter ...
  const uint64_t* iter_ptr;    // ... or read from device memory when non-null
  int mode_k;
  int reject_cap;
  int64_t det_cap;             // candidate-product cap
  int64_t det_buf;             // capacity of the deterministic key buffer
};

// Buffers of one sampling pass (device), sized by sample_buffers_bytes.
struct SampleBuffers {
  SampleState* state;
  uint32_t* cand;       // sum_t n_t candidate indices (mode t at cand_off[t])
  int64_t cand_off[kMaxOrder];
  uint64_t* det_keys;   // det_cap packed keys
  double* det_p;        // det_cap probabilities
  uint64_t* sortA;      // s: per-slot random keys of the draws, then the sort input
  uint64_t* sortB;      // s
  uint64_t* hkeys;      // 2^hbits combine-table keys
  uint32_t* hcnt;       // 2^hbits repeat counts
  int hbits;
  char* scratch;        // max(sort, scan) workspace for s items
  // outputs
  uint64_t* idx_packed; // s
  uint32_t* cnt;        // s
  double* wgt;          // s
  uint64_t* idx_linear; // s (may be null)
  uint64_t* raw_key;    // s_rnd raw per-slot linear keys (may be null)
  double* raw_w;        // s_rnd raw per-slot weights (may be null)
};

size_t sample_buffers_bytes(const KeyLayout& L, int64_t s, int64_t det_buf);
void sample_buffers_carve(Arena& a, const KeyLayout& L, int64_t s, int64_t det_buf,
                          SampleBuffers* B);

// Deterministic-buffer capacity for a pass: s suffices when tau * s >= 1, because
// then fewer than 1/tau <= s rows can have p > tau.
int64_t det_buffer_capacity(int64_t s, double tau, int64_t det_cap);

// Enqueue one SkrpLev pass.  If tau * s < 1 the deterministic set might exceed s;
// then the call synchronises once to run the top-s selection (never the case when
// tau * s >= 1, so that path is free of host synchronisation).  sorted_output:
// rows in the order of Alg. 1's cat (deterministic keys ascending, then random
// keys ascending); otherwise rows come in table order, which the solve does not
// depend on.
int skrp_lev(const SampleParams& P, SampleBuffers& B, cudaStream_t st, bool sorted_output);

}  // namespace cpa
