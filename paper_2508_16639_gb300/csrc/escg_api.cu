// escg_api.cu -- the C ABI of libescg (include/escg.h): handle life cycle,
// host-side set-up (partition tables, integer rate thresholds, transition
// table, the initial lattice) and run orchestration on the handle's stream.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <vector>

#include "escg.h"
#include "escg_diag.h"
#include "escg_internal.h"

using namespace escg_impl;

namespace {

thread_local char g_err[512] = "";

void set_err(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

}  // namespace

void escg_impl::set_last_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

namespace {

#define CUDA_TRY(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      set_err("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return ESCG_ECUDA;                                                                \
    }                                                                                   \
  } while (0)

constexpr uint32_t kDefaultSpinLimit = 2000000;  // polls of ~1 us: a few seconds
// Largest number of generic block-owner CTAs per SM that persistent = 1
// accepts.
constexpr int kGownDefaultPerSM = 3;
// Blocks per coarse phase over 256-thread flag-kernel CTAs from which
// persistent = 1 runs the flag kernel's 128-thread build.
constexpr int kFlag128Ratio = 3;

// Schedule v1 partition of one axis (both axes are identical).
struct Partition {
  int P = 0, GQ = 0;
  std::vector<int32_t> cs, fs, fc;
};

void split_even(int n, int parts, int32_t* start) {
  const int q = n / parts, r = n % parts;
  start[0] = 0;
  for (int k = 0; k < parts; ++k) start[k + 1] = start[k] + q + (k < r ? 1 : 0);
}

Partition make_partition(int L) {
  Partition p;
  const int h = (L + 64) / 128;
  p.P = 2 * (h < 1 ? 1 : h);
  p.cs.resize(p.P + 1);
  split_even(L, p.P, p.cs.data());
  p.fc.resize(p.P + 1);
  for (int k = 0; k < p.P; ++k) {
    const int w = p.cs[k + 1] - p.cs[k];
    const int Q = 2 * (w / 4);
    std::vector<int32_t> loc(Q + 1);
    split_even(w, Q, loc.data());
    p.fc[k] = (int)p.fs.size();
    for (int q = 0; q < Q; ++q) p.fs.push_back(p.cs[k] + loc[q]);
  }
  p.GQ = (int)p.fs.size();
  p.fc[p.P] = p.GQ;
  p.fs.push_back(L);
  return p;
}

// 2-D uint8 tensor map of a lattice for the TMA tile loads: dims L x L
// (columns beyond L are out of bounds and read as zero), row stride pitch,
// box 112 x 66 bytes.
bool make_tensor_map(CUtensorMap* map, uint8_t* lattice, int L, int pitch) {
  return encode_lattice_map(map, lattice, L, pitch, 112, 66);
}

}  // namespace

bool escg_impl::encode_lattice_map(CUtensorMap* map, uint8_t* lattice, int L, int pitch, int box_w,
                                   int box_h) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)L, (cuuint64_t)L};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  const cuuint32_t elem[2] = {1u, 1u};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, lattice, dims, strides, box, elem,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

// The closed form (AxisGeom) reproduces the partition tables, and every fine
// segment is 2..4 sites wide (the kernels' reciprocal table covers those).
bool axis_geom_matches(const AxisGeom& g, const Partition& p) {
  for (int b = 0; b < p.P; ++b) {
    const bool wide = b < g.r;
    const int nw = b < g.r ? b : g.r;
    const int s0 = b * g.q + nw, w = g.q + (wide ? 1 : 0);
    const int f0 = nw * g.Qa + (b - nw) * g.Qb, Q = wide ? g.Qa : g.Qb;
    const int fq = wide ? g.fqa : g.fqb, fr = wide ? g.fra : g.frb;
    if (p.cs[b] != s0 || p.cs[b + 1] - p.cs[b] != w || p.fc[b] != f0 || p.fc[b + 1] - p.fc[b] != Q) return false;
    for (int k = 0; k < Q; ++k) {
      const int st = k * fq + (k < fr ? k : fr), wk = fq + (k < fr ? 1 : 0);
      if (p.fs[f0 + k] != s0 + st || wk < 2 || wk > 4) return false;
    }
  }
  return true;
}

bool partition_fits(const Partition& p) {
  for (int k = 0; k < p.P; ++k) {
    if (p.cs[k + 1] - p.cs[k] > kMaxBlock) return false;
    if (p.fc[k + 1] - p.fc[k] > kMaxFine) return false;
  }
  return true;
}

bool thresholds(const escg_rates* r, uint64_t* tx, uint64_t* txi) {
  const double I = r->interact, Pr = r->reproduce, X = r->exchange;
  if (!(I >= 0.0) || !(Pr >= 0.0) || !(X >= 0.0)) return false;
  const double R = (X + I) + Pr;
  if (!(R > 0.0) || std::isinf(R)) return false;
  *tx = (uint64_t)std::floor(std::ldexp(X / R, 32) + 0.5);
  *txi = (uint64_t)std::floor(std::ldexp((X + I) / R, 32) + 0.5);
  return true;
}

}  // namespace

namespace escg_impl {

// Transition table (LatticeDesc::trans) of Alg. 3 for every (action,
// selected a, neighbour b): exchange swaps distinct values; interaction
// empties the dominated one (selected site tested first; empty sites never
// dominate, Alg. 2); reproduction copies the selected species into an empty
// neighbour or the neighbour's species into an empty selected site; action 3
// changes nothing.  Interaction thresholds: an edge with probability p
// (Park, Chen and Szolnoki) takes place iff u < T_X + round((T_XI - T_X) q /
// 2^32), q = round(p 2^32) -- exact integer arithmetic, so the value does not
// depend on the compiler's floating-point contraction; prob == nullptr
// means every edge is certain (T_XI).
void build_transitions(int S, const uint8_t* D, const double* prob, uint64_t tx, uint64_t txi,
                       uint32_t* out) {
  const int s1 = S + 1;
  std::memset(out, 0, sizeof(uint32_t) * kTransWords);
  uint8_t* t = reinterpret_cast<uint8_t*>(out);
  auto dom = [&](int x, int y) { return x != 0 && y != 0 && D[(x - 1) * S + (y - 1)] == 1; };
  for (int act = 0; act < 4; ++act)
    for (int a = 0; a < s1; ++a)
      for (int b = 0; b < s1; ++b) {
        int na = a, nb = b;
        if (a != b) {
          if (act == 0) {
            na = b;
            nb = a;
          } else if (act == 1) {
            if (dom(a, b))
              nb = 0;
            else if (dom(b, a))
              na = 0;
          } else if (act == 2) {
            if (b == 0)
              nb = a;
            else if (a == 0)
              na = b;
          }
        }
        t[(a * s1 + b) * 4 + act] = (uint8_t)(na | (nb << 4));
      }
  for (int a = 0; a < s1; ++a)
    for (int b = 0; b < s1; ++b) {
      double p = 1.0;
      if (prob && a != 0 && b != 0 && a != b) {
        if (dom(a, b))
          p = prob[(a - 1) * S + (b - 1)];
        else if (dom(b, a))
          p = prob[(b - 1) * S + (a - 1)];
      }
      uint64_t tp = txi;
      if (!(p > 0.0)) {
        tp = tx;
      } else if (p < 1.0) {
        const uint64_t q = (uint64_t)std::floor(std::ldexp(p, 32) + 0.5);
        const unsigned __int128 w = (unsigned __int128)(txi - tx) * q + ((unsigned __int128)1 << 31);
        tp = tx + (uint64_t)(w >> 32);
      }
      out[kTransPairs + a * s1 + b] = (tp >> 32) ? 0xFFFFFFFFu : (uint32_t)tp;
    }
}

}  // namespace escg_impl

struct escg {
  int device = 0;
  int L = 0, H = 0, S = 0, pitch = 0;   // columns, rows, species, row stride
  uint64_t seed = 0;
  escg_options opt{};
  Partition part, part_y;               // column and row partitions
  LatticeDesc desc{};
  cudaStream_t stream = nullptr;
  bool own_stream = false, own_lattice = false;
  uint8_t* lattice = nullptr;
  int32_t* d_tables = nullptr;   // cs | fs | fc, then the row axis's (if H != L)
  uint8_t* d_trans = nullptr;
  RunState* d_state = nullptr;
  unsigned long long* d_log = nullptr;
  uint32_t* d_log_mcs = nullptr;
  uint32_t* d_done = nullptr;    // P*Py absolute epochs of the persistent kernel
  unsigned long long* d_ob = nullptr;  // boundary records of the mailbox kernel
  bool use_ll = false;           // uniform geometry, plain persistent path
  uint64_t mcs_enq = 0;          // MCS number after all enqueued work
  uint64_t launches = 0;
  uint64_t T_empty = 0;
  int grid = 0;
  bool use_tma = false;
  bool use_resident = false;     // persistent = 4 and the lattice fits one CTA's shared memory
  bool use_own = false;          // block-owner kernel (uniform, square, one byte per site)
  int own_dyn = 0;               // its shared-memory padding
  int own_threads = 0;           // and CTA size
  int flag_threads = 256;        // CTA size of the flag kernel (128: uniform geometry, > 4 CTAs per SM)
  bool use_gown = false;         // block owners on a generic partition
  int tuned_mode = 0, tuned_ctas = 0;   // autotuner's choice (launch mode, CTAs per SM)
  double tuned_ms_per_mcs = 0.0;
  int tuned_candidates = 0;      // configurations timed (0: taken from the cache)
  GownConfig gown{};
  size_t ob_words = 0;           // boundary-record words allocated (all blocks)
  CUtensorMap tmap{};
  uint32_t spin_limit = kDefaultSpinLimit;
  int stall_block = -1;
  uint32_t log_num0_host = 0;
  bool failed = false;
  RunState* d_scratch = nullptr;  // accumulator for on-demand counts
  uint32_t* h_err = nullptr;      // pinned word: error bits of an asynchronous host step
  bool pending_step = false;      // an escg_step_host_async has not been waited for
  int bits = 8;                   // bits per site of the device lattice
  uint8_t* d_stage = nullptr;     // packed lattices: byte image for host transfers
  int stage_pitch = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_free;
  double kernel_ms = 0.0;
  uint64_t kernel_launches = 0;
};

namespace {

LogBuffers log_buffers(escg* h) { return LogBuffers{h->d_log, h->d_log_mcs}; }

// Byte image of a packed lattice for host transfers (allocated on first use).
cudaError_t ensure_stage(escg* h) {
  if (h->d_stage) return cudaSuccess;
  h->stage_pitch = escg_lattice_pitch(h->L);
  return cudaMalloc(&h->d_stage, (size_t)h->H * h->stage_pitch);
}

// The lattice as one byte per site: the device lattice itself, or the byte
// image of a packed one.
LatticeDesc byte_view(escg* h) {
  LatticeDesc d = h->desc;
  if (h->bits != 8) {
    d.lat = h->d_stage;
    d.pitch = h->stage_pitch;
    d.bits = 8;
  }
  return d;
}

// Host <-> device copy of the H x L lattice (host rows packed, device rows of
// the handle's pitch); one linear copy when the two layouts coincide.  A
// packed lattice goes through its byte image and the pack / unpack kernels.
cudaError_t copy_to_device(escg* h, const uint8_t* host) {
  if (h->bits != 8) {
    cudaError_t e = ensure_stage(h);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(h->d_stage, h->stage_pitch, host, h->L, h->L, h->H, cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess) e = launch_pack(h->desc, h->d_stage, h->stage_pitch, h->stream);
    return e;
  }
  if (h->pitch == h->L)
    return cudaMemcpyAsync(h->lattice, host, (size_t)h->L * h->H, cudaMemcpyHostToDevice, h->stream);
  return cudaMemcpy2DAsync(h->lattice, h->pitch, host, h->L, h->L, h->H, cudaMemcpyHostToDevice, h->stream);
}
cudaError_t copy_to_host(escg* h, uint8_t* host) {
  if (h->bits != 8) {
    cudaError_t e = ensure_stage(h);
    if (e == cudaSuccess) e = launch_unpack(h->desc, h->d_stage, h->stage_pitch, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(host, h->L, h->d_stage, h->stage_pitch, h->L, h->H, cudaMemcpyDeviceToHost,
                            h->stream);
    return e;
  }
  if (h->pitch == h->L)
    return cudaMemcpyAsync(host, h->lattice, (size_t)h->L * h->H, cudaMemcpyDeviceToHost, h->stream);
  return cudaMemcpy2DAsync(host, h->L, h->lattice, h->pitch, h->L, h->H, cudaMemcpyDeviceToHost, h->stream);
}

int enqueue_log(escg* h, uint32_t m_end, bool log, uint64_t check_total = 0) {
  if (log) {
    CUDA_TRY(launch_count(h->desc, h->d_state, h->stream));
    h->launches++;
  }
  CUDA_TRY(launch_finalize(h->desc, h->d_state, log_buffers(h), m_end, h->opt.log_every, log ? 1 : 0,
                           h->opt.stop_at_extinction, h->stream, check_total));
  h->launches++;
  return ESCG_OK;
}

// Optional CUDA-event bracketing of the lattice-update launches.
cudaError_t timing_begin(escg* h) {
  if (!h->opt.time_kernels) return cudaSuccess;
  if (h->ev_free.empty()) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    h->ev_free.emplace_back(a, b);
  }
  h->ev_used.push_back(h->ev_free.back());
  h->ev_free.pop_back();
  return cudaEventRecord(h->ev_used.back().first, h->stream);
}

cudaError_t timing_end(escg* h) {
  if (!h->opt.time_kernels) return cudaSuccess;
  return cudaEventRecord(h->ev_used.back().second, h->stream);
}

// Device-side reset of the run state to MCS `mcs` (no host memory is read
// asynchronously, so nothing waits here).  validate: the lattice was just
// replaced; its bytes are checked (0..S, else the run state stops with
// kErrBadValue) -- by the count of MCS mcs when that is a log point of a
// one-byte lattice (the counts must add up to L*H), else by the validate
// kernel.
int reset_state(escg* h, uint64_t mcs, bool validate = false) {
  const uint32_t le = h->opt.log_every;
  const uint32_t num0 = (uint32_t)((mcs + le - 1) / le);
  CUDA_TRY(launch_state_reset(h->d_state, (uint32_t)mcs, num0, h->stream));
  h->launches++;
  CUDA_TRY(launch_fill_u32(h->d_done, h->part.P * h->part_y.P, (uint32_t)mcs, h->stream));
  h->launches++;
  // Boundary records left by an earlier run carry epochs the new one may wait
  // for (a lattice restored at an MCS the handle has run through before):
  // epoch 0 never matches a wait, which always expects an epoch >= 1.
  if (h->d_ob) CUDA_TRY(cudaMemsetAsync(h->d_ob, 0, h->ob_words * sizeof(unsigned long long), h->stream));
  h->log_num0_host = num0;
  h->mcs_enq = mcs;
  h->failed = false;
  const bool log = mcs % h->opt.log_every == 0;
  const bool by_count = validate && log && h->bits == 8;
  if (log) {
    const int rc = enqueue_log(h, (uint32_t)mcs, true, by_count ? (uint64_t)h->L * h->H : 0);
    if (rc != ESCG_OK) return rc;
  }
  if (validate && !by_count) {
    CUDA_TRY(launch_validate(byte_view(h), &h->d_state->error, kErrBadValue, &h->d_state->stopped, h->stream));
    h->launches++;
  }
  return ESCG_OK;
}

void free_handle(escg* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->own_lattice && h->lattice) cudaFree(h->lattice);
  cudaFree(h->d_tables);
  cudaFree(h->d_stage);
  if (h->h_err) cudaFreeHost(h->h_err);
  cudaFree(h->d_trans);
  cudaFree(h->d_state);
  cudaFree(h->d_log);
  cudaFree(h->d_log_mcs);
  cudaFree(h->d_done);
  cudaFree(h->d_ob);
  cudaFree(h->d_scratch);
  for (auto& e : h->ev_used) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& e : h->ev_free) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// Boundary records of at least `words` words (zeroed by the next reset).
int ensure_records(escg* h, size_t words) {
  if (h->ob_words >= words) return ESCG_OK;
  cudaFree(h->d_ob);
  h->d_ob = nullptr;
  h->ob_words = 0;
  if (cudaMalloc(&h->d_ob, words * sizeof(unsigned long long)) != cudaSuccess) {
    set_err("cudaMalloc of %zu boundary-record bytes failed", words * sizeof(unsigned long long));
    return ESCG_ENOMEM;
  }
  h->ob_words = words;
  return ESCG_OK;
}

// Picks the lattice-update kernel for launch mode `persistent` (escg_options)
// and the CTAs per SM of the ticketed kernels (0: as many as fit), from the
// partition, the storage and the device's occupancy.  Physical mapping only:
// every choice gives the same lattices.
int select_kernel(escg* h, int persistent, int ctas_per_sm) {
  LatticeDesc& d = h->desc;
  const Partition& p = h->part;
  const Partition& py = h->part_y;
  const int L = h->L, H = h->H;
  h->use_tma = h->use_ll = h->use_own = h->use_gown = h->use_resident = false;
  h->own_dyn = h->own_threads = 0;
  h->gown = GownConfig{};
  h->grid = persistent_grid(h->device, d.uniform64 != 0 || d.uniform_var != 0);
  // the TMA and mailbox kernels are written for square lattices of one byte
  // per site; the flag kernel takes rectangular and packed ones in both
  // geometries
  const bool square = (H == L) && h->bits == 8;
  if (d.uniform64 && square && persistent == 2) {
    if (!make_tensor_map(&h->tmap, h->lattice, L, h->pitch)) {
      set_err("cuTensorMapEncodeTiled failed for L=%d", L);
      return ESCG_ECUDA;
    }
    h->use_tma = true;
    h->grid = persistent_tma_grid(h->device);
  }
  // The mailbox kernel shortens every hop of the colour-phase chain but
  // binds each CTA's next item one visit early.  Measured (GB300, 608 CTAs):
  // faster than the flag kernel while a coarse phase has at most half as
  // many blocks as there are CTAs (L <= 2048: 10-25 %), slower with 576 or
  // 625 blocks per phase (L = 3072, 3200: 3-5 %), where the flag kernel keeps
  // items unbound until a CTA is free.  It runs on request (6) and by default
  // where the block owners below cannot.
  if (d.uniform64 && square && (persistent == 1 || persistent == 6) &&
      (persistent == 6 || 2 * (p.P * p.P / 4) <= persistent_ll_grid(h->device))) {
    if (ensure_records(h, (size_t)p.P * p.P * kRecordWords) != ESCG_OK) return ESCG_ENOMEM;
    h->use_ll = true;
    h->grid = persistent_ll_grid(h->device);
  }
  // Block owners: on request (5), and by default (1) from 3 x 3 groups of
  // blocks while the grid needs at most 3 CTAs per SM -- measured (GB300, µs
  // per MCS, mailbox or flag kernel vs owners): L = 384 15.4 vs 14.1, 512
  // 15.9 vs 14.4, 1024 18.2 vs 13.0, 1536 20.0 vs 12.4, 2048 19.7 vs 15.1,
  // 2560 23.3 vs 19.5; tied at L = 256 and at 4 per SM (3072); slower at
  // L = 128 (13.3 vs 14.0) and from 5 per SM (3200: 25.5 vs 29.2), where every
  // CTA of an SM is in the same colour phase at once and the flag kernel's
  // free binding keeps the SMs busier.  Needs the device to hold one CTA per
  // 2x2 group of blocks at once.
  if (d.uniform64 && (persistent == 5 || (persistent == 1 && (p.P / 2) * (py.P / 2) >= 9))) {
    int dyn = 0, nt = 0, per_sm = 0;
    if (persistent_own_config(d, h->device, &dyn, &nt, &per_sm, ctas_per_sm) > 0 &&
        (persistent == 5 || per_sm <= 3)) {
      if (ensure_records(h, (size_t)p.P * py.P * kRecordWords) != ESCG_OK) return ESCG_ENOMEM;
      h->use_own = true;
      h->own_dyn = dyn;
      h->own_threads = nt;
      h->use_ll = false;
    }
  }
  // Block owners on a generic partition (von Neumann rule, periodic or
  // reflecting, any bits per site): on request (5), and by default (1) from
  // 2 x 2 groups of blocks while the grid needs at most kGownDefaultPerSM
  // CTAs per SM.  Needs the device to hold one CTA per group at once.
  if (!d.uniform64 && d.nbh == 4 &&
      (persistent == 5 || (persistent == 1 && (p.P / 2) * (py.P / 2) >= 2))) {
    GownConfig cfg{};
    if (persistent_gown_config(d, h->device, &cfg, ctas_per_sm) > 0 &&
        (persistent == 5 || cfg.ctas_per_sm <= kGownDefaultPerSM)) {
      if (ensure_records(h, (size_t)p.P * py.P * kGRecordWords) != ESCG_OK) return ESCG_ENOMEM;
      h->use_gown = true;
      h->gown = cfg;
    }
  }
  // Whole-lattice residency: on request (4), and by default (1) for a generic
  // partition with 2 x 2 coarse blocks (L, H < 192 and not 128), where it was
  // measured 1.4-2.2x faster than the flag kernel's dependency chain of
  // generic visits (tied at L = 200, slower beyond; the mailbox kernel is
  // faster for the uniform L = 128).
  if ((persistent == 4 || (persistent == 1 && !d.uniform64 && p.P == 2 && py.P == 2)) &&
      resident_fits(d, h->device)) {
    h->use_resident = true;
    h->use_gown = false;
  }
  // The flag kernel on a uniform lattice (any bits per site) with more than
  // 4 CTAs per SM requested, or by default (1) with at least kFlag128Ratio times as many
  // blocks per coarse phase as 256-thread CTAs: the 128-thread build (two
  // quads per thread), up to 8 per SM.  Measured (µs per MCS, 4 x 256 vs
  // 8 x 128 threads per SM): L = 2048 21.7 vs 26.7, 3200 25.5 vs 32.8 (5 x 128:
  // 28.9), 6400 91.4 vs 78.7 -- more visits in flight pay once the phases are
  // several waves deep and throughput, not the colour chain, binds.
  h->flag_threads = 256;
  const bool flag = !h->use_tma && !h->use_ll && !h->use_own && !h->use_gown && !h->use_resident;
  const bool deep = persistent == 1 && (int64_t)p.P * py.P / 4 >= (int64_t)kFlag128Ratio * h->grid;
  if (flag && (ctas_per_sm > 4 || deep) && d.uniform64) {
    h->flag_threads = 128;
    h->grid = persistent_grid128(h->device);
  }
  if (ctas_per_sm > 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (sms * ctas_per_sm < h->grid) h->grid = sms * ctas_per_sm;
  }

  return ESCG_OK;
}

int check_inputs(int32_t L, int32_t S, const uint8_t* D, const escg_rates* rates) {
  if (L < 8 || L > 16384) {
    set_err("L=%d out of range [8, 16384]", L);
    return ESCG_EINVAL;
  }
  if (S < 2 || S > 15) {
    set_err("S=%d out of range [2, 15]", S);
    return ESCG_EINVAL;
  }
  if (!D || !rates) {
    set_err("digraph and rates must not be NULL");
    return ESCG_EINVAL;
  }
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) {
      if (D[i * S + j] > 1) {
        set_err("digraph[%d][%d]=%d is not 0 or 1", i, j, D[i * S + j]);
        return ESCG_EINVAL;
      }
      if (i == j && D[i * S + j]) {
        set_err("digraph has a nonzero diagonal at %d", i);
        return ESCG_EINVAL;
      }
    }
  uint64_t tx, txi;
  if (!thresholds(rates, &tx, &txi)) {
    set_err("rates must be finite, >= 0 and not all zero");
    return ESCG_EINVAL;
  }
  return ESCG_OK;
}

}  // namespace

extern "C" {

void escg_default_options(escg_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->p_empty = 0.0;
  opt->log_every = 10;
  opt->stop_at_extinction = 0;
  opt->schedule_version = 1;
  opt->persistent = 1;
}

int32_t escg_lattice_pitch(int32_t L) { return L <= 0 ? 0 : ((L + 15) / 16) * 16; }

size_t escg_lattice_bytes(int32_t L) { return L <= 0 ? 0 : (size_t)L * escg_lattice_pitch(L); }

size_t escg_lattice_bytes_rect(int32_t L, int32_t H) {
  return (L <= 0 || H <= 0) ? 0 : (size_t)H * escg_lattice_pitch(L);
}

int32_t escg_lattice_pitch_ex(int32_t L, int32_t bits_per_site) {
  if (bits_per_site == 0) bits_per_site = 8;
  if (L <= 0 || (bits_per_site != 8 && bits_per_site != 4 && bits_per_site != 2)) return 0;
  const int64_t bytes = ((int64_t)L * bits_per_site + 7) / 8;
  return (int32_t)((bytes + 15) / 16 * 16);
}

size_t escg_lattice_bytes_ex(int32_t L, int32_t H, int32_t bits_per_site) {
  return H <= 0 ? 0 : (size_t)H * escg_lattice_pitch_ex(L, bits_per_site);
}

const char* escg_last_error(void) { return g_err; }

double escg_exchange_from_mobility(double M, int64_t N) { return 2.0 * M * (double)N; }

int escg_circulant(int32_t S, const int32_t* K, int32_t nK, uint8_t* D) {
  if (S < 1 || nK < 0 || (nK > 0 && !K) || !D) {
    set_err("bad circulant arguments");
    return ESCG_EINVAL;
  }
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) {
      const int off = ((j - i) % S + S) % S;
      uint8_t v = 0;
      for (int k = 0; k < nK; ++k) v |= (uint8_t)(off == K[k]);
      D[i * S + j] = v;
    }
  return ESCG_OK;
}

}  // extern "C"
static int autotune(escg* h);
extern "C" {

escg_t* escg_create(int32_t L, int32_t S, const uint8_t* digraph, const escg_rates* rates, uint64_t seed) {
  escg_options o;
  escg_default_options(&o);
  return escg_create_ex(L, S, digraph, rates, seed, &o);
}

escg_t* escg_create_ex(int32_t L, int32_t S, const uint8_t* digraph, const escg_rates* rates,
                       uint64_t seed, const escg_options* opt) {
  g_err[0] = 0;
  if (check_inputs(L, S, digraph, rates) != ESCG_OK) return nullptr;
  escg_options o;
  escg_default_options(&o);
  if (opt) o = *opt;
  if (o.log_every == 0) o.log_every = 10;
  if (o.dominance_prob) {
    for (int k = 0; k < S * S; ++k)
      if (!(o.dominance_prob[k] >= 0.0 && o.dominance_prob[k] <= 1.0)) {
        set_err("dominance_prob[%d] is not in [0,1]", k);
        return nullptr;
      }
  }
  if (o.neighbourhood == 0) o.neighbourhood = 4;
  if ((o.neighbourhood != 4 && o.neighbourhood != 8) || (o.reflecting_boundary != 0 && o.reflecting_boundary != 1)) {
    set_err("neighbourhood must be 4 or 8 and reflecting_boundary 0 or 1");
    return nullptr;
  }
  if (o.height == 0) o.height = L;
  if (o.height < 8 || o.height > 16384) {
    set_err("height=%d out of range [8, 16384]", o.height);
    return nullptr;
  }
  if (o.bits_per_site == 0) o.bits_per_site = 8;
  if (o.bits_per_site != 8 && o.bits_per_site != 4 && o.bits_per_site != 2) {
    set_err("bits_per_site must be 8, 4 or 2 (got %d)", o.bits_per_site);
    return nullptr;
  }
  if (o.bits_per_site == 2 && S > 3) {
    set_err("2 bits per site hold the values 0..3: S=%d needs 4 or 8", S);
    return nullptr;
  }
  if (o.bits_per_site != 8 && (L < 64 || o.height < 64)) {
    set_err("a packed lattice needs L, H >= 64 (blocks at least 32 sites wide), got %d x %d", L, o.height);
    return nullptr;
  }
  if (reinterpret_cast<uintptr_t>(o.device_lattice) % 16 != 0) {
    set_err("device_lattice must be 16-byte aligned (rows are read as 16-byte vectors)");
    return nullptr;
  }
  if (o.autotune != 0 && o.autotune != 1) {
    set_err("autotune must be 0 or 1 (got %d)", o.autotune);
    return nullptr;
  }
  if (o.persistent < 0 || o.persistent > 6) {
    set_err("persistent must be 0..6 (got %d)", o.persistent);
    return nullptr;
  }
  if (o.schedule_version != 0 && o.schedule_version != 1) {
    set_err("schedule_version %u is not supported (only 1)", o.schedule_version);
    return nullptr;
  }
  if (!(o.p_empty >= 0.0 && o.p_empty <= 1.0)) {
    set_err("p_empty=%g outside [0, 1]", o.p_empty);
    return nullptr;
  }
  escg* h = new (std::nothrow) escg;
  if (!h) {
    set_err("host allocation failed");
    return nullptr;
  }
  const int H = o.height;
  h->L = L;
  h->H = H;
  h->S = S;
  h->seed = seed;
  h->opt = o;
  h->bits = o.bits_per_site;
  h->pitch = escg_lattice_pitch_ex(L, h->bits);
  h->part = make_partition(L);
  h->part_y = make_partition(H);
  if (!partition_fits(h->part) || !partition_fits(h->part_y)) {
    set_err("internal: partition of %d x %d exceeds the kernel's block limits", L, H);
    delete h;
    return nullptr;
  }
  h->T_empty = (uint64_t)std::floor(std::ldexp(o.p_empty, 32) + 0.5);

  auto fail = [&](int code) -> escg_t* {
    (void)code;
    free_handle(h);
    return nullptr;
  };
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    set_err("no CUDA device available (libescg has no CPU fallback)");
    return fail(ESCG_ECUDA);
  }
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    set_err("cudaGetDevice failed");
    return fail(ESCG_ECUDA);
  }

  cudaError_t e = cudaSuccess;
  if (o.cuda_stream) {
    h->stream = (cudaStream_t)o.cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    h->own_stream = true;
  }
  const size_t nbytes = escg_lattice_bytes_ex(L, H, h->bits);
  if (e == cudaSuccess) {
    if (o.device_lattice) {
      h->lattice = (uint8_t*)o.device_lattice;
    } else {
      e = cudaMalloc(&h->lattice, nbytes);
      h->own_lattice = true;
    }
  }
  const Partition& p = h->part;
  const Partition& py = h->part_y;
  const size_t ntab_x = p.cs.size() + p.fs.size() + p.fc.size();
  const size_t ntab = ntab_x + (H != L ? py.cs.size() + py.fs.size() + py.fc.size() : 0);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_tables, ntab * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_trans, sizeof(uint32_t) * kTransWords);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_state, sizeof(RunState));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_log, sizeof(unsigned long long) * kLogCap * kMaxStates);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_log_mcs, sizeof(uint32_t) * kLogCap);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_done, sizeof(uint32_t) * p.P * py.P);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_scratch, sizeof(RunState));
  if (e != cudaSuccess) {
    set_err("device allocation failed: %s", cudaGetErrorString(e));
    return fail(ESCG_ENOMEM);
  }
  std::vector<int32_t> tab;
  tab.insert(tab.end(), p.cs.begin(), p.cs.end());
  tab.insert(tab.end(), p.fs.begin(), p.fs.end());
  tab.insert(tab.end(), p.fc.begin(), p.fc.end());
  if (H != L) {
    tab.insert(tab.end(), py.cs.begin(), py.cs.end());
    tab.insert(tab.end(), py.fs.begin(), py.fs.end());
    tab.insert(tab.end(), py.fc.begin(), py.fc.end());
  }
  uint64_t tx = 0, txi = 0;
  thresholds(rates, &tx, &txi);
  std::vector<uint32_t> trans(kTransWords);
  build_transitions(S, digraph, o.dominance_prob, tx, txi, trans.data());
  if (cudaMemcpyAsync(h->d_tables, tab.data(), tab.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                      h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->d_trans, trans.data(), trans.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    set_err("upload of lattice tables failed");
    return fail(ESCG_ECUDA);
  }
  LatticeDesc& d = h->desc;
  d.lat = h->lattice;
  d.L = L;
  d.pitch = h->pitch;
  d.P = p.P;
  d.GQ = p.GQ;
  d.cs = h->d_tables;
  d.fs = h->d_tables + p.cs.size();
  d.fc = h->d_tables + p.cs.size() + p.fs.size();
  d.H = H;
  d.Py = py.P;
  d.csy = H != L ? h->d_tables + ntab_x : d.cs;
  d.fsy = H != L ? d.csy + py.cs.size() : d.fs;
  d.fcy = H != L ? d.fsy + py.fs.size() : d.fc;
  d.ax = make_axis_geom(L, p.P);
  d.ay = make_axis_geom(H, py.P);
  d.bits = h->bits;
  if (!axis_geom_matches(d.ax, p) || !axis_geom_matches(d.ay, py)) {
    set_err("internal: closed-form partition disagrees with the tables for %d x %d", L, H);
    return fail(ESCG_EINVAL);
  }
  d.trans = h->d_trans;
  d.key0 = (uint32_t)seed;
  d.key1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    d.rk[2 * r] = d.key0 + (uint32_t)r * 0x9E3779B9u;
    d.rk[2 * r + 1] = d.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  // 2^32 ("always") becomes 0xFFFFFFFF: exact, since every action draw u
  // is a multiple of 4 and so never equals 0xFFFFFFFF
  d.tx = tx >> 32 ? 0xFFFFFFFFu : (uint32_t)tx;
  d.txi = txi >> 32 ? 0xFFFFFFFFu : (uint32_t)txi;
  d.S = S;
  fill_perm24(d.perm24);
  bool uni = true;
  for (int k = 0; k < p.P; ++k) uni = uni && (p.cs[k + 1] - p.cs[k] == 64);
  for (int k = 0; k < p.GQ; ++k) uni = uni && (p.fs[k + 1] - p.fs[k] == 2);
  for (int k = 0; k < py.P; ++k) uni = uni && (py.cs[k + 1] - py.cs[k] == 64);
  for (int k = 0; k < py.GQ; ++k) uni = uni && (py.fs[k + 1] - py.fs[k] == 2);
  d.nbh = o.neighbourhood;
  d.reflect = o.reflecting_boundary;
  // the uniform kernels implement the von Neumann, periodic rule; the flag
  // kernel also the variants on 64 x 64 blocks of one byte per site
  d.uniform64 = (uni && h->pitch % 16 == 0 && d.nbh == 4 && !d.reflect) ? 1 : 0;
  d.uniform_var = (uni && h->pitch % 16 == 0 && (d.nbh == 8 || d.reflect) && h->bits == 8) ? 1 : 0;
  if (select_kernel(h, o.persistent, o.ctas_per_sm) != ESCG_OK) return fail(ESCG_ENOMEM);

  if (launch_init(d, h->T_empty, h->stream) != cudaSuccess) {
    set_err("init kernel launch failed");
    return fail(ESCG_ECUDA);
  }
  h->launches++;
  if (reset_state(h, 0) != ESCG_OK) return fail(ESCG_ECUDA);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    set_err("initialisation failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(ESCG_ECUDA);
  }
  if (o.autotune && o.persistent == 1 && autotune(h) != ESCG_OK) return fail(ESCG_ECUDA);
  return h;
}

int escg_run(escg_t* h, uint64_t n_mcs) {
  if (!h) {
    set_err("NULL handle");
    return ESCG_EINVAL;
  }
  if (h->failed) {
    set_err("handle is in an error state; restore a lattice first");
    return ESCG_ESTATE;
  }
  const uint64_t target = h->mcs_enq + n_mcs;
  if (target > 0xFFFFFFFFull) {
    set_err("MCS number would exceed 2^32-1");
    return ESCG_EINVAL;
  }
  const uint32_t k = h->opt.log_every;
  // rule variants count log points with the count kernel between launches
  // (the resident kernel counts in-kernel for every rule)
  const bool fused = (h->desc.nbh == 4 && !h->desc.reflect) || h->use_resident;
  while (h->mcs_enq < target) {
    uint64_t end;
    if (h->opt.persistent && !h->opt.stop_at_extinction && fused) {
      // one launch may leave up to kPendRing log points open
      const uint64_t lim = (h->mcs_enq / k + kPendRing) * k;
      end = lim < target ? lim : target;
    } else {
      // stasis is decided at log points: a launch ends there
      const uint64_t next_log = (h->mcs_enq / k + 1) * k;
      end = next_log < target ? next_log : target;
    }
    // the persistent kernel numbers work items with 32-bit tickets
    const uint64_t per_mcs = (uint64_t)h->part.P * h->part_y.P;
    const uint64_t max_chunk = ((1ull << 31) - (uint64_t)h->grid) / per_mcs;
    if (end - h->mcs_enq > max_chunk) end = h->mcs_enq + max_chunk;
    const uint32_t m0 = (uint32_t)h->mcs_enq, n = (uint32_t)(end - h->mcs_enq);
    if (h->opt.persistent) {
      const uint64_t items = (uint64_t)n * per_mcs;
      const int grid = (int)(items < (uint64_t)h->grid ? items : (uint64_t)h->grid);
      PersistentArgs a{};
      a.d = h->desc;
      a.st = h->d_state;
      a.done = h->d_done;
      a.lb = log_buffers(h);
      a.m_begin = m0;
      a.n_mcs = n;
      a.log_every = k;
      a.stop_at_extinction = h->opt.stop_at_extinction;
      a.spin_limit = h->spin_limit;
      a.stall_block = h->stall_block;
      a.ob = h->d_ob;
      a.fuse_counts = fused ? 1 : 0;
      a.threads = h->flag_threads;
      CUDA_TRY(timing_begin(h));
      if (h->use_resident) {
        CUDA_TRY(launch_resident(a, h->stream));
      } else if (h->use_own) {
        CUDA_TRY(launch_persistent_own(a, h->own_dyn, h->own_threads, h->stream));
      } else if (h->use_gown) {
        CUDA_TRY(launch_persistent_gown(a, h->gown, h->stream));
      } else if (h->use_tma) {
        TmaArgs ta{};
        ta.map = h->tmap;
        ta.p = a;
        CUDA_TRY(launch_persistent_tma(ta, grid, h->stream));
      } else if (h->use_ll) {
        CUDA_TRY(launch_persistent_ll(a, grid, h->stream));
      } else {
        CUDA_TRY(launch_persistent(a, grid, h->stream));
      }
      CUDA_TRY(timing_end(h));
      h->launches++;
      if (h->use_ll) {
        CUDA_TRY(launch_ll_merge(h->desc, h->d_ob, h->d_state, (uint32_t)end, h->stream));
        h->launches++;
      }
      if (fused) {
        h->mcs_enq = end;
        continue;  // counts of log points and the MCS number are written in-kernel
      }
    } else {
      for (uint32_t m = m0; m < m0 + n; ++m)
        for (int slot = 0; slot < 4; ++slot) {
          CUDA_TRY(timing_begin(h));
          CUDA_TRY(launch_phase(h->desc, h->d_state, m, slot, h->stream));
          CUDA_TRY(timing_end(h));
          h->launches++;
        }
    }
    h->mcs_enq = end;
    const int rc = enqueue_log(h, (uint32_t)end, end % k == 0);
    if (rc != ESCG_OK) return rc;
  }
  return ESCG_OK;
}

int escg_sync(escg_t* h) {
  if (!h) {
    set_err("NULL handle");
    return ESCG_EINVAL;
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  RunState st;
  CUDA_TRY(cudaMemcpy(&st, h->d_state, sizeof st, cudaMemcpyDeviceToHost));
  if (st.error & kErrTimeout) {
    h->failed = true;
    set_err("a bounded device-side wait timed out; the lattice is inconsistent until restored");
    return ESCG_ETIMEOUT;
  }
  return ESCG_OK;
}

int escg_counts(escg_t* h, uint64_t* out, uint64_t* mcs_out) {
  if (!h || !out) {
    set_err("NULL argument");
    return ESCG_EINVAL;
  }
  int rc = escg_sync(h);
  if (rc != ESCG_OK) return rc;
  // separate scratch state so the run's accumulator is untouched
  RunState* tmp = h->d_scratch;
  cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(RunState), h->stream);
  if (e == cudaSuccess) e = launch_count(h->desc, tmp, h->stream);
  h->launches++;
  RunState st{}, cur{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cur, tmp, sizeof cur, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, h->d_state, sizeof st, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    set_err("count failed: %s", cudaGetErrorString(e));
    return ESCG_ECUDA;
  }
  for (int v = 0; v <= h->S; ++v) out[v] = cur.cur[v];
  if (mcs_out) *mcs_out = st.mcs;
  return ESCG_OK;
}

int escg_counts_log(escg_t* h, uint64_t* out, uint64_t* mcs_out, int64_t cap, int64_t* n_out) {
  if (!h || (!out && cap > 0) || cap < 0) {
    set_err("bad arguments");
    return ESCG_EINVAL;
  }
  int rc = escg_sync(h);
  if (rc != ESCG_OK) return rc;
  RunState st;
  CUDA_TRY(cudaMemcpy(&st, h->d_state, sizeof st, cudaMemcpyDeviceToHost));
  const int64_t have = st.n_log < (uint32_t)kLogCap ? st.n_log : kLogCap;
  const int64_t n = have < cap ? have : cap;
  std::vector<unsigned long long> buf((size_t)kLogCap * kMaxStates);
  std::vector<uint32_t> ms(kLogCap);
  CUDA_TRY(cudaMemcpy(buf.data(), h->d_log, buf.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(ms.data(), h->d_log_mcs, ms.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  const uint32_t first = st.n_log - (uint32_t)have;  // oldest retained entry
  for (int64_t i = 0; i < n; ++i) {
    const uint32_t idx = (first + (uint32_t)i) % (uint32_t)kLogCap;
    for (int v = 0; v <= h->S; ++v) out[i * (h->S + 1) + v] = buf[(size_t)idx * kMaxStates + v];
    if (mcs_out) mcs_out[i] = ms[idx];
  }
  if (n_out) *n_out = n;
  return ESCG_OK;
}

int escg_snapshot(escg_t* h, uint8_t* host_out) {
  if (!h || !host_out) {
    set_err("NULL argument");
    return ESCG_EINVAL;
  }
  int rc = escg_sync(h);
  if (rc != ESCG_OK) return rc;
  CUDA_TRY(copy_to_host(h, host_out));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return ESCG_OK;
}

int escg_restore(escg_t* h, const uint8_t* host_lattice, uint64_t mcs) {
  if (!h || !host_lattice) {
    set_err("NULL argument");
    return ESCG_EINVAL;
  }
  if (mcs > 0xFFFFFFFFull) {
    set_err("mcs exceeds 2^32-1");
    return ESCG_EINVAL;
  }
  CUDA_TRY(copy_to_device(h, host_lattice));
  // values are checked on the device; an invalid lattice also stops the
  // run state, so that nothing enqueued later touches it
  const int rc = reset_state(h, mcs, true);
  if (rc != ESCG_OK) return rc;
  uint32_t err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, &h->d_state->error, sizeof err, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (err & kErrBadValue) {
    h->failed = true;
    set_err("restored lattice holds a value outside 0..S=%d; restore a valid lattice", h->S);
    return ESCG_EINVAL;
  }
  return ESCG_OK;
}

// Enqueues the whole host step (restore, run, snapshot, counts) and the copy
// of the run state's error bits to the handle's pinned word; nothing waits.
static int step_host_enqueue(escg* h, const uint8_t* host_in, uint64_t mcs, uint64_t n_mcs, uint8_t* host_out,
                      uint64_t* counts_out) {
  if (!h || !host_in || !host_out) {
    set_err("NULL argument");
    return ESCG_EINVAL;
  }
  if (mcs > 0xFFFFFFFFull) {
    set_err("mcs exceeds 2^32-1");
    return ESCG_EINVAL;
  }
  if (!h->h_err && cudaMallocHost(&h->h_err, sizeof(uint32_t)) != cudaSuccess) {
    h->h_err = nullptr;
    set_err("pinned host allocation failed");
    return ESCG_ENOMEM;
  }
  // copy in, reset, check (an invalid lattice stops the run state on the
  // device), run, copy out, counts, error bits
  CUDA_TRY(copy_to_device(h, host_in));
  int rc = reset_state(h, mcs, true);
  if (rc != ESCG_OK) return rc;
  rc = escg_run(h, n_mcs);
  if (rc != ESCG_OK) return rc;
  CUDA_TRY(copy_to_host(h, host_out));
  if (counts_out) {
    const uint64_t end = mcs + n_mcs, le = h->opt.log_every;
    if (!h->opt.stop_at_extinction && end % le == 0 && end / le >= h->log_num0_host) {
      // the run logged the counts of its final MCS: read that entry
      const uint64_t slot = (end / le - h->log_num0_host) % (uint64_t)kLogCap;
      CUDA_TRY(cudaMemcpyAsync(counts_out, h->d_log + slot * kMaxStates, sizeof(uint64_t) * (h->S + 1),
                               cudaMemcpyDeviceToHost, h->stream));
    } else {
      CUDA_TRY(cudaMemsetAsync(h->d_scratch, 0, sizeof(RunState), h->stream));
      CUDA_TRY(launch_count(h->desc, h->d_scratch, h->stream));
      h->launches++;
      CUDA_TRY(cudaMemcpyAsync(counts_out, h->d_scratch->cur, sizeof(uint64_t) * (h->S + 1),
                               cudaMemcpyDeviceToHost, h->stream));
    }
  }
  CUDA_TRY(cudaMemcpyAsync(h->h_err, &h->d_state->error, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
  h->pending_step = true;
  return ESCG_OK;
}

int escg_step_host_wait(escg_t* h) {
  if (!h) {
    set_err("NULL handle");
    return ESCG_EINVAL;
  }
  if (!h->pending_step) return ESCG_OK;
  h->pending_step = false;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  const uint32_t err = *h->h_err;
  if (err & kErrBadValue) {
    h->failed = true;
    set_err("input lattice holds a value outside 0..S=%d", h->S);
    return ESCG_EINVAL;
  }
  if (err & kErrTimeout) {
    h->failed = true;
    set_err("a bounded device-side wait timed out; the lattice is inconsistent until restored");
    return ESCG_ETIMEOUT;
  }
  return ESCG_OK;
}

int escg_step_host_async(escg_t* h, const uint8_t* host_in, uint64_t mcs, uint64_t n_mcs, uint8_t* host_out,
                         uint64_t* counts_out) {
  if (h && h->pending_step) {
    set_err("a host step is already in flight on this handle; wait for it first");
    return ESCG_ESTATE;
  }
  return step_host_enqueue(h, host_in, mcs, n_mcs, host_out, counts_out);
}

int escg_step_host(escg_t* h, const uint8_t* host_in, uint64_t mcs, uint64_t n_mcs, uint8_t* host_out,
                   uint64_t* counts_out) {
  // one synchronisation for the whole call
  if (h && h->pending_step) {
    const int rc = escg_step_host_wait(h);
    if (rc != ESCG_OK) return rc;
  }
  const int rc = step_host_enqueue(h, host_in, mcs, n_mcs, host_out, counts_out);
  if (rc != ESCG_OK) return rc;
  return escg_step_host_wait(h);
}

void* escg_device_lattice(escg_t* h) { return h ? (void*)h->lattice : nullptr; }
void* escg_stream(escg_t* h) { return h ? (void*)h->stream : nullptr; }
uint64_t escg_launch_count(escg_t* h) { return h ? h->launches : 0; }

uint64_t escg_current_mcs(escg_t* h) {
  if (!h) return 0;
  if (escg_sync(h) != ESCG_OK) return 0;
  RunState st;
  if (cudaMemcpy(&st, h->d_state, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
  return st.mcs;
}

int escg_kernel_time(escg_t* h, double* ms_total, uint64_t* n_launches, int reset) {
  if (!h) {
    set_err("NULL handle");
    return ESCG_EINVAL;
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (auto& e : h->ev_used) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e.first, e.second));
    h->kernel_ms += ms;
    h->kernel_launches++;
    h->ev_free.push_back(e);
  }
  h->ev_used.clear();
  if (ms_total) *ms_total = h->kernel_ms;
  if (n_launches) *n_launches = h->kernel_launches;
  if (reset) {
    h->kernel_ms = 0.0;
    h->kernel_launches = 0;
  }
  return ESCG_OK;
}

int escg_debug_stall_block(escg_t* h, int32_t block, uint32_t spin_limit) {
  if (!h) {
    set_err("NULL handle");
    return ESCG_EINVAL;
  }
  if (block >= h->part.P * h->part_y.P) {
    set_err("block %d out of range", block);
    return ESCG_EINVAL;
  }
  h->stall_block = block < 0 ? -1 : block;
  h->spin_limit = spin_limit ? spin_limit : kDefaultSpinLimit;
  return ESCG_OK;
}

int32_t escg_coarse_blocks(escg_t* h) { return h ? h->part.P : 0; }

const char* escg_update_kernel(escg_t* h) {
  if (!h) return "";
  if (!h->opt.persistent) return "phase_kernel";
  if (h->use_resident) return "resident_kernel";
  if (h->use_own) return "persistent_own_kernel";
  if (h->use_gown) return "persistent_gown_kernel";
  if (h->use_tma) return "persistent_tma_kernel";
  return h->use_ll ? "persistent_ll_kernel" : "persistent_kernel";
}

void escg_destroy(escg_t* h) { free_handle(h); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner.  Every launch mode and CTA count gives the same lattice, so the
// fastest is a measured, result-neutral choice.  On the first handle of a
// (device, L, H, S, bits per site, rule) the candidates are timed on a
// scratch copy of the initial lattice -- 10 MCS to warm up, then 20 MCS
// between two CUDA events -- and the winner is cached for the process; the
// handle then starts from its initial lattice at MCS 0 as if just created.
namespace {

struct TuneKey {
  int dev, L, H, S, bits, nbh, reflect;
  bool operator<(const TuneKey& o) const {
    const int a[7] = {dev, L, H, S, bits, nbh, reflect}, b[7] = {o.dev, o.L, o.H, o.S, o.bits, o.nbh, o.reflect};
    for (int i = 0; i < 7; ++i)
      if (a[i] != b[i]) return a[i] < b[i];
    return false;
  }
};
struct TuneVal {
  int mode, ctas;
  double ms_per_mcs;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

// What a selection runs, for dropping candidates that duplicate another.
std::string kernel_signature(escg* h) {
  char buf[128];
  snprintf(buf, sizeof buf, "%s/%d/%d/%d/%d", escg_update_kernel(h), h->grid, h->own_threads, h->gown.threads,
           h->flag_threads);
  return buf;
}

// Device time of 20 MCS of the current selection from the scratch lattice
// (after 10 MCS of warm-up), or a negative value if a wait timed out.
int tune_time(escg* h, const uint8_t* scratch, size_t nbytes, double* ms) {
  CUDA_TRY(cudaMemcpyAsync(h->lattice, scratch, nbytes, cudaMemcpyDeviceToDevice, h->stream));
  int rc = reset_state(h, 0);
  if (rc == ESCG_OK) rc = escg_run(h, 10);
  if (rc != ESCG_OK) return rc;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  cudaEventRecord(e0, h->stream);
  rc = escg_run(h, 20);
  cudaEventRecord(e1, h->stream);
  if (rc == ESCG_OK) rc = escg_sync(h);
  float t = 0.f;
  if (rc == ESCG_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = ESCG_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = rc == ESCG_OK ? (double)t : -1.0;
  return rc == ESCG_ETIMEOUT ? ESCG_OK : rc;   // a timed-out candidate only loses
}

}  // namespace

static int autotune(escg* h) {
  const TuneKey key{h->device, h->L, h->H, h->S, h->bits, h->desc.nbh, h->desc.reflect};
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it != g_tune.end()) {
    h->tuned_mode = it->second.mode;
    h->tuned_ctas = it->second.ctas;
    h->tuned_ms_per_mcs = it->second.ms_per_mcs;
    h->tuned_candidates = 0;
    return select_kernel(h, it->second.mode, it->second.ctas);
  }
  const size_t nbytes = escg_lattice_bytes_ex(h->L, h->H, h->bits);
  uint8_t* scratch = nullptr;
  if (cudaMalloc(&scratch, nbytes) != cudaSuccess) {
    set_err("autotune: cudaMalloc of a %zu-byte scratch lattice failed", nbytes);
    return ESCG_ENOMEM;
  }
  CUDA_TRY(cudaMemcpyAsync(scratch, h->lattice, nbytes, cudaMemcpyDeviceToDevice, h->stream));
  const int saved_timing = h->opt.time_kernels, saved_stop = h->opt.stop_at_extinction;
  h->opt.time_kernels = 0;
  h->opt.stop_at_extinction = 0;
  // (launch mode, CTAs per SM of the ticketed kernels): the default rule,
  // the flag kernel at 4, 3 and 2 CTAs per SM and (128-thread CTAs) 8 and 6,
  // the mailbox kernel at 4 and 3,
  // the TMA-staged flag kernel, the block owners, whole-lattice residency;
  // modes a lattice cannot run fall back to one already listed and are
  // dropped as duplicates
  const int cand[][2] = {{1, 0}, {3, 0}, {3, 3}, {3, 2}, {3, 8}, {3, 6}, {6, 0}, {6, 3}, {2, 0}, {5, 0}, {4, 0}};
  std::vector<std::string> seen;
  int best_mode = 1, best_ctas = 0, n = 0, rc = ESCG_OK;
  double best = -1.0;
  for (const auto& c : cand) {
    rc = select_kernel(h, c[0], c[1]);
    if (rc != ESCG_OK) break;
    const std::string sig = kernel_signature(h);
    bool dup = false;
    for (const auto& x : seen) dup = dup || x == sig;
    if (dup) continue;
    seen.push_back(sig);
    double ms = -1.0;
    rc = tune_time(h, scratch, nbytes, &ms);
    if (rc != ESCG_OK) break;
    ++n;
    if (ms >= 0.0 && (best < 0.0 || ms < best)) {
      best = ms;
      best_mode = c[0];
      best_ctas = c[1];
    }
  }
  h->opt.time_kernels = saved_timing;
  h->opt.stop_at_extinction = saved_stop;
  if (rc == ESCG_OK) rc = select_kernel(h, best_mode, best_ctas);
  if (rc == ESCG_OK) {
    cudaError_t e = cudaMemcpyAsync(h->lattice, scratch, nbytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) rc = reset_state(h, 0);
    if (e == cudaSuccess && rc == ESCG_OK) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      set_err("autotune: restoring the initial lattice failed: %s", cudaGetErrorString(e));
      rc = ESCG_ECUDA;
    }
  }
  cudaFree(scratch);
  if (rc != ESCG_OK) return rc;
  h->tuned_mode = best_mode;
  h->tuned_ctas = best_ctas;
  h->tuned_ms_per_mcs = best / 20.0;
  h->tuned_candidates = n;
  g_tune[key] = TuneVal{best_mode, best_ctas, best / 20.0};
  return ESCG_OK;
}

extern "C" int escg_autotune_result(escg_t* h, int32_t* persistent, int32_t* ctas_per_sm, double* ms_per_mcs,
                                    int32_t* candidates) {
  if (!h) {
    set_err("NULL handle");
    return ESCG_EINVAL;
  }
  if (!h->opt.autotune) {
    set_err("the handle was not created with autotune");
    return ESCG_ESTATE;
  }
  if (persistent) *persistent = h->tuned_mode;
  if (ctas_per_sm) *ctas_per_sm = h->tuned_ctas;
  if (ms_per_mcs) *ms_per_mcs = h->tuned_ms_per_mcs;
  if (candidates) *candidates = h->tuned_candidates;
  return ESCG_OK;
}
