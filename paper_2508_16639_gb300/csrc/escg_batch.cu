// escg_batch.cu -- batched ensembles (include/escg.h, escg_batch_*): many
// independent replicas of uneven L in shared persistent launches.
//
// Device layout: one arena holds every replica's lattice, partition tables,
// transition table and block epochs; SlotDesc (static, per replica) and
// SlotState (dynamic) arrays describe them.  A run is a sequence of chunks of
// log_every MCS.  Each chunk is two kernels on the batch's stream:
//   batch_compact_kernel  advances every active replica's MCS by the last
//                         chunk, retires replicas that went extinct or spent
//                         their budget, admits new ones, and rebuilds the
//                         work table (one entry per block of a coarse phase
//                         of every active replica);
//   batch_kernel          persistent: CTAs take work items (chunk MCS index,
//                         coarse slot, table entry) from a ticket counter, wait
//                         for the block's 8 neighbours in its own replica
//                         (bounded spin), and visit the block exactly as the
//                         single-lattice kernels do; the counts of the chunk's
//                         final MCS (a log point) are fused in, and the last
//                         block of a replica decides its stasis.
// The chunk sequence needs no host round trip, so it is captured once in a
// CUDA graph and replayed.  A replica's trajectory depends only on its own
// parameters: items of different replicas never share data.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "escg.h"
#include "escg_device.cuh"
#include "escg_internal.h"

namespace escg_impl {

struct SlotDesc {
  LatticeDesc d;
  uint32_t* done;       // [P*P] absolute epochs
  uint32_t max_mcs;     // budget: absolute MCS number to stop at
  int32_t stop_at_extinction;
  int32_t nb4;          // blocks per coarse phase = P*P/4
  int32_t pad;
};

struct SlotState {
  uint32_t mcs;         // absolute MCS reached (advanced by the compaction)
  uint32_t stopped;     // stasis reached
  uint32_t pend;        // blocks done at the open log point
  uint32_t counts_mcs;  // MCS of `counts`
  unsigned long long acc[kMaxStates];
  unsigned long long counts[kMaxStates];   // counts at the last log point
};

struct BatchCtl {
  uint32_t n_active, tot4, chunk, ticket;
  uint32_t exited, error, abort, n_admit;
  uint32_t last_chunk;  // MCS the previous batch_kernel launch covered
  uint32_t pad[7];
};

struct BatchArgs {
  const SlotDesc* slots;
  SlotState* states;
  BatchCtl* ctl;
  const uint32_t* table;   // (slot << 16) | block-of-phase
  uint32_t log_every;
  uint32_t spin_limit;
};

__device__ __forceinline__ uint32_t b_ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void b_st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t b_ld_volatile(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

// Counts of the whole lattice of every slot (one CTA per slot), written as
// the slot's log entry of its current MCS; sets stopped when <= 1 species
// is alive and the slot stops at extinction.  Used once, at creation/admission.
__global__ void batch_count_kernel(const SlotDesc* slots, SlotState* states, const uint32_t* which, int n) {
  const int w = blockIdx.x;
  if (w >= n) return;
  const int s = which ? (int)which[w] : w;
  const LatticeDesc& d = slots[s].d;
  __shared__ uint32_t hist[kMaxStates];
  if (threadIdx.x < kMaxStates) hist[threadIdx.x] = 0;
  __syncthreads();
  const int L = d.L, pitch = d.pitch;
  for (int k = threadIdx.x; k < L * L; k += blockDim.x) {
    const int r = k / L, c = k - r * L;
    atomicAdd(&hist[d.lat[(size_t)r * pitch + c]], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    SlotState& st = states[s];
    int alive = 0;
    for (int v = 0; v < kMaxStates; ++v) {
      const unsigned long long c = (v <= d.S) ? hist[v] : 0ull;
      st.counts[v] = c;
      st.acc[v] = 0;
      if (v >= 1 && v <= d.S && c > 0) ++alive;
    }
    st.counts_mcs = st.mcs;
    st.pend = 0;
    if (slots[s].stop_at_extinction && alive <= 1) st.stopped = 1;
  }
}

// Single CTA.  Advances the active replicas by the last chunk, retires the
// finished ones, admits the slots listed in `admit`, and rebuilds the work
// table and the launch control block for the next chunk.
constexpr int kCompactThreads = 1024;
__global__ void __launch_bounds__(kCompactThreads) batch_compact_kernel(const SlotDesc* slots, SlotState* states,
                                                                        BatchCtl* ctl, uint32_t* active,
                                                                        uint32_t* active_tmp, uint32_t* table,
                                                                        const uint32_t* admit, uint32_t chunk) {
  __shared__ uint32_t s_scan[kCompactThreads];
  __shared__ uint32_t s_keep_total, s_n_old, s_n_admit, s_last;
  const int t = threadIdx.x;
  if (t == 0) {
    s_n_old = ctl->n_active;
    s_n_admit = ctl->n_admit;
    s_last = ctl->last_chunk;
  }
  __syncthreads();
  const uint32_t n_old = s_n_old, n_admit = s_n_admit, last = s_last;
  const uint32_t n_all = n_old + n_admit;
  // 1. advance and decide which slots stay (old active first, then admitted)
  const uint32_t per = (n_all + kCompactThreads - 1) / kCompactThreads;
  const uint32_t lo = t * per, hi = min(n_all, lo + per);
  uint32_t keep_count = 0;
  for (uint32_t a = lo; a < hi; ++a) {
    const uint32_t s = a < n_old ? active[a] : admit[a - n_old];
    SlotState& st = states[s];
    if (a < n_old && !st.stopped) {
      const uint32_t nm = st.mcs + last;
      st.mcs = nm < slots[s].max_mcs ? nm : slots[s].max_mcs;
    } else if (a < n_old && st.stopped) {
      st.mcs = st.counts_mcs;
    }
    if (!st.stopped && st.mcs < slots[s].max_mcs) ++keep_count;
  }
  s_scan[t] = keep_count;
  __syncthreads();
  for (int off = 1; off < kCompactThreads; off <<= 1) {   // inclusive scan
    const uint32_t v = t >= off ? s_scan[t - off] : 0u;
    __syncthreads();
    s_scan[t] += v;
    __syncthreads();
  }
  uint32_t pos = s_scan[t] - keep_count;
  if (t == kCompactThreads - 1) s_keep_total = s_scan[t];
  for (uint32_t a = lo; a < hi; ++a) {
    const uint32_t s = a < n_old ? active[a] : admit[a - n_old];
    const SlotState& st = states[s];
    if (!st.stopped && st.mcs < slots[s].max_mcs) active_tmp[pos++] = s;
  }
  __syncthreads();
  const uint32_t n_new = s_keep_total;
  // 2. work table: nb4 entries per kept slot, in active order
  const uint32_t per2 = (n_new + kCompactThreads - 1) / kCompactThreads;
  const uint32_t lo2 = t * per2, hi2 = min(n_new, lo2 + per2);
  uint32_t sum = 0;
  for (uint32_t a = lo2; a < hi2; ++a) sum += (uint32_t)slots[active_tmp[a]].nb4;
  __syncthreads();
  s_scan[t] = sum;
  __syncthreads();
  for (int off = 1; off < kCompactThreads; off <<= 1) {
    const uint32_t v = t >= off ? s_scan[t - off] : 0u;
    __syncthreads();
    s_scan[t] += v;
    __syncthreads();
  }
  uint32_t e = s_scan[t] - sum;
  for (uint32_t a = lo2; a < hi2; ++a) {
    const uint32_t s = active_tmp[a];
    active[a] = s;
    const uint32_t nb4 = (uint32_t)slots[s].nb4;
    for (uint32_t j = 0; j < nb4; ++j) table[e++] = (s << 16) | j;
  }
  __syncthreads();
  if (t == kCompactThreads - 1) {
    ctl->n_active = n_new;
    ctl->tot4 = s_scan[t];
    ctl->chunk = chunk;
    ctl->ticket = 0;
    ctl->exited = 0;
    ctl->n_admit = 0;
    ctl->last_chunk = 0;   // consumed; the next batch_kernel launch sets it
  }
}

// Persistent multi-replica chunk kernel.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) batch_kernel(BatchArgs a) {
  __shared__ VisitSmem sm;
  __shared__ SlotDesc sd;
  __shared__ uint32_t s_quit, s_skip, s_abort, s_slot, s_m, s_ord;
  __shared__ int32_t s_k, s_bx, s_by, s_col;
  BatchCtl* ctl = a.ctl;
  const int tid = threadIdx.x;
  const uint32_t tot4 = ctl->tot4, chunk = ctl->chunk;
  const uint64_t total = (uint64_t)chunk * 4u * tot4;
  for (;;) {
    if (tid == 0) {
      const uint32_t t = atomicAdd(&ctl->ticket, 1u);
      uint32_t quit = ((uint64_t)t >= total) || b_ld_volatile(&ctl->abort);
      if (!quit) {
        const uint32_t i = t / (4u * tot4), rem = t - i * 4u * tot4;
        const uint32_t k = rem / tot4, e = a.table[rem - k * tot4];
        s_slot = e >> 16;
        s_k = (int32_t)k;
        s_m = i;   // chunk-relative for now
        s_by = (int32_t)(e & 0xFFFFu);   // block index within the phase
      }
      s_quit = quit;
      s_abort = 0;
    }
    if (tid < kMaxStates) sm.hist[tid] = 0;
    __syncthreads();
    if (s_quit) break;
    {  // the replica's descriptor
      const uint32_t* src = reinterpret_cast<const uint32_t*>(a.slots + s_slot);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sd);
      for (int w = tid; w < (int)(sizeof(SlotDesc) / 4); w += THREADS) dst[w] = src[w];
    }
    __syncthreads();
    const LatticeDesc& d = sd.d;
    if (tid == 0) {
      const uint32_t m = a.states[s_slot].mcs + s_m;
      s_m = m;
      s_skip = m >= sd.max_mcs;
      if (!s_skip) {
        const uint32_t ord = colour_order(philox10_rk(make_uint4(0u, 0u, m, kTagOrder), d.rk).x, d.perm24);
        const int colour = order_at(ord, s_k), j = s_by, half = d.P >> 1;
        s_ord = ord;
        s_col = colour;
        s_bx = 2 * (j % half) + (colour & 1);
        s_by = 2 * (j / half) + (colour >> 1);
      }
    }
    load_trans(d, sm.trans);
    __syncthreads();
    if (s_skip) continue;   // beyond this replica's budget
    const uint32_t m = s_m, ord = s_ord;
    const int k = s_k, colour = s_col, bx = s_bx, by = s_by, P = d.P;
    if (tid < 9) {
      const int dx = tid % 3 - 1, dy = tid / 3 - 1;
      const int nx = (bx + dx + P) % P, ny = (by + dy + P) % P;
      const int ncol = colour ^ ((dx & 1) | ((dy & 1) << 1));
      const uint32_t need = (tid == 4) ? m : (slot_of(ord, ncol) < k ? m + 1u : m);
      const uint32_t* flag = sd.done + ny * P + nx;
      uint32_t spins = 0;
      while (b_ld_acquire(flag) < need) {
        if (b_ld_volatile(&ctl->abort)) {
          s_abort = 1;
          break;
        }
        if (++spins > a.spin_limit) {
          atomicOr(&ctl->error, kErrTimeout);
          atomicExch(&ctl->abort, 1u);
          s_abort = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __syncthreads();
    if (s_abort) break;
    visit_generic(d, bx, by, m, sm);
    const bool log_point = ((m + 1u) % a.log_every) == 0u;
    if (log_point) {
      const int sV = slot_of(ord, colour ^ 2), sH = slot_of(ord, colour ^ 1), sD = slot_of(ord, colour ^ 3);
      count_visit_generic(d, bx, by, sm, k, sV, sH, sD);
    }
    __syncthreads();
    if (log_point) {
      SlotState* st = a.states + s_slot;
      if (tid <= d.S && sm.hist[tid]) atomicAdd(&st->acc[tid], (unsigned long long)sm.hist[tid]);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        if (atomicAdd(&st->pend, 1u) == (uint32_t)(P * P) - 1u) {
          __threadfence();
          int alive = 0;
          for (int v = 0; v < kMaxStates; ++v) {
            const unsigned long long c = atomicExch(&st->acc[v], 0ull);
            st->counts[v] = c;
            if (v >= 1 && v <= d.S && c > 0) ++alive;
          }
          st->counts_mcs = m + 1u;
          st->pend = 0;
          if (sd.stop_at_extinction && alive <= 1) st->stopped = 1;
        }
      }
    }
    if (tid == 0) {
      __threadfence();
      b_st_release(sd.done + by * P + bx, m + 1u);
    }
  }
  // the last CTA to leave records how far this launch advanced the replicas
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&ctl->exited, 1u) == gridDim.x - 1u) {
      ctl->exited = 0;
      ctl->last_chunk = chunk;
    }
  }
}

}  // namespace escg_impl

using namespace escg_impl;

namespace {

#define bset_err set_last_error

struct BPartition {
  int P = 0, GQ = 0;
  std::vector<int32_t> cs, fs, fc;
};

void bsplit(int n, int parts, int32_t* start) {
  const int q = n / parts, r = n % parts;
  start[0] = 0;
  for (int k = 0; k < parts; ++k) start[k + 1] = start[k] + q + (k < r ? 1 : 0);
}

BPartition bpartition(int L) {
  BPartition p;
  const int h = (L + 64) / 128;
  p.P = 2 * (h < 1 ? 1 : h);
  p.cs.resize(p.P + 1);
  bsplit(L, p.P, p.cs.data());
  p.fc.resize(p.P + 1);
  for (int k = 0; k < p.P; ++k) {
    const int w = p.cs[k + 1] - p.cs[k], Q = 2 * (w / 4);
    std::vector<int32_t> loc(Q + 1);
    bsplit(w, Q, loc.data());
    p.fc[k] = (int)p.fs.size();
    for (int q = 0; q < Q; ++q) p.fs.push_back(p.cs[k] + loc[q]);
  }
  p.GQ = (int)p.fs.size();
  p.fc[p.P] = p.GQ;
  p.fs.push_back(L);
  return p;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct escg_batch {
  int n = 0;
  int device = 0;
  escg_batch_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint8_t* arena = nullptr;
  SlotDesc* d_slots = nullptr;
  SlotState* d_states = nullptr;
  BatchCtl* d_ctl = nullptr;
  uint32_t* d_active = nullptr;
  uint32_t* d_active_tmp = nullptr;
  uint32_t* d_table = nullptr;
  uint32_t* d_admit = nullptr;
  std::vector<SlotDesc> h_slots;
  std::vector<int> L, S;
  int threads = 0;          // CTA size in use (0: not tuned yet)
  int grid[3] = {0, 0, 0};  // persistent grid per CTA size 64/128/256
  uint64_t launches = 0;
  uint64_t mcs_budget_max = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_chunks = 0;
  uint32_t* h_nactive = nullptr;  // pinned
  uint32_t spin_limit = 2000000;
};

namespace {

int tsel(int threads) { return threads == 64 ? 0 : (threads == 128 ? 1 : 2); }

cudaError_t launch_batch_kernel(escg_batch* b, int threads) {
  BatchArgs a{b->d_slots, b->d_states, b->d_ctl, b->d_table, b->opt.log_every, b->spin_limit};
  const int g = b->grid[tsel(threads)];
  if (threads == 64)
    batch_kernel<64><<<g, 64, 0, b->stream>>>(a);
  else if (threads == 128)
    batch_kernel<128><<<g, 128, 0, b->stream>>>(a);
  else
    batch_kernel<256><<<g, 256, 0, b->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_compact(escg_batch* b) {
  batch_compact_kernel<<<1, kCompactThreads, 0, b->stream>>>(b->d_slots, b->d_states, b->d_ctl, b->d_active,
                                                             b->d_active_tmp, b->d_table, b->d_admit,
                                                             b->opt.log_every);
  return cudaGetLastError();
}

// one chunk: compaction (retire / advance) then the persistent work kernel
cudaError_t enqueue_chunk(escg_batch* b, int threads) {
  cudaError_t e = launch_compact(b);
  if (e != cudaSuccess) return e;
  b->launches += 2;
  return launch_batch_kernel(b, threads);
}

void free_batch(escg_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->arena);
  cudaFree(b->d_slots);
  cudaFree(b->d_states);
  cudaFree(b->d_ctl);
  cudaFree(b->d_active);
  cudaFree(b->d_active_tmp);
  cudaFree(b->d_table);
  cudaFree(b->d_admit);
  if (b->h_nactive) cudaFreeHost(b->h_nactive);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int active_count(escg_batch* b, uint32_t* out) {
  if (cudaMemcpyAsync(b->h_nactive, &b->d_ctl->n_active, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    bset_err("reading the active count failed");
    return ESCG_ECUDA;
  }
  *out = *b->h_nactive;
  return ESCG_OK;
}

}  // namespace

extern "C" {

void escg_batch_default_options(escg_batch_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->log_every = 10;
  opt->threads = 0;
  opt->use_graph = 1;
}

escg_batch_t* escg_batch_create(int32_t n, const escg_replica_spec* specs, const escg_batch_options* opt) {
  if (n < 1 || n > 65535 || !specs) {
    bset_err("need 1 <= n <= 65535 replicas");
    return nullptr;
  }
  escg_batch* b = new (std::nothrow) escg_batch;
  if (!b) return nullptr;
  b->n = n;
  escg_batch_default_options(&b->opt);
  if (opt) b->opt = *opt;
  if (b->opt.log_every == 0) b->opt.log_every = 10;
  if (b->opt.threads != 0 && b->opt.threads != 64 && b->opt.threads != 128 && b->opt.threads != 256) {
    bset_err("threads must be 0, 64, 128 or 256");
    free_batch(b);
    return nullptr;
  }
  b->threads = b->opt.threads;
  // host image of the arena: per replica lattice | tables | trans | done
  struct Off { size_t lat, tab, trans, done; BPartition part; uint64_t TE; };
  std::vector<Off> off(n);
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    const escg_replica_spec& sp = specs[i];
    // validation (shared rules with escg_create)
    escg_options o;
    escg_default_options(&o);
    if (sp.L < 8 || sp.L > 16384 || sp.S < 2 || sp.S > 15 || !sp.digraph) {
      bset_err("replica %d: bad L=%d / S=%d / digraph", i, sp.L, sp.S);
      free_batch(b);
      return nullptr;
    }
    for (int a = 0; a < sp.S * sp.S; ++a)
      if (sp.digraph[a] > 1 || (a / sp.S == a % sp.S && sp.digraph[a])) {
        bset_err("replica %d: digraph must be 0/1 with a zero diagonal", i);
        free_batch(b);
        return nullptr;
      }
    const double I = sp.rates.interact, Pr = sp.rates.reproduce, X = sp.rates.exchange;
    if (!(I >= 0 && Pr >= 0 && X >= 0) || !((X + I) + Pr > 0) || std::isinf((X + I) + Pr) ||
        !(sp.p_empty >= 0.0 && sp.p_empty <= 1.0) || sp.max_mcs > 0xFFFFFFFFull) {
      bset_err("replica %d: bad rates / p_empty / max_mcs", i);
      free_batch(b);
      return nullptr;
    }
    Off& f = off[i];
    f.part = bpartition(sp.L);
    for (int k = 0; k < f.part.P; ++k)
      if (f.part.cs[k + 1] - f.part.cs[k] > kMaxBlock) {
        bset_err("replica %d: partition exceeds block limits", i);
        free_batch(b);
        return nullptr;
      }
    const int pitch = escg_lattice_pitch(sp.L);
    f.lat = total;
    total = align_up(total + (size_t)sp.L * pitch, 256);
    f.tab = total;
    total = align_up(total + 4 * (f.part.cs.size() + f.part.fs.size() + f.part.fc.size()), 256);
    f.trans = total;
    total = align_up(total + 4 * (size_t)(sp.S + 1) * (sp.S + 1), 256);
    f.done = total;
    total = align_up(total + 4 * (size_t)f.part.P * f.part.P, 256);
    f.TE = (uint64_t)std::floor(std::ldexp(sp.p_empty, 32) + 0.5);
    b->L.push_back(sp.L);
    b->S.push_back(sp.S);
    if (sp.max_mcs > b->mcs_budget_max) b->mcs_budget_max = sp.max_mcs;
  }
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) {
    if (b->opt.cuda_stream) {
      b->stream = (cudaStream_t)b->opt.cuda_stream;
    } else {
      e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
      b->own_stream = true;
    }
  }
  size_t table_cap = 0;
  for (int i = 0; i < n; ++i) table_cap += (size_t)off[i].part.P * off[i].part.P / 4;
  if (e == cudaSuccess) e = cudaMalloc(&b->arena, total);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_slots, sizeof(SlotDesc) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_states, sizeof(SlotState) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, sizeof(BatchCtl));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_active, sizeof(uint32_t) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_active_tmp, sizeof(uint32_t) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_table, sizeof(uint32_t) * table_cap);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_admit, sizeof(uint32_t) * n);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_nactive, sizeof(uint32_t));
  if (e != cudaSuccess) {
    bset_err("batch allocation failed: %s", cudaGetErrorString(e));
    free_batch(b);
    return nullptr;
  }
  std::vector<uint8_t> image(total, 0);
  b->h_slots.resize(n);
  for (int i = 0; i < n; ++i) {
    const escg_replica_spec& sp = specs[i];
    const Off& f = off[i];
    const BPartition& p = f.part;
    int32_t* tab = reinterpret_cast<int32_t*>(image.data() + f.tab);
    size_t w = 0;
    for (int32_t v : p.cs) tab[w++] = v;
    for (int32_t v : p.fs) tab[w++] = v;
    for (int32_t v : p.fc) tab[w++] = v;
    // transition table of Alg. 3 (same layout as the single-lattice path)
    const int s1 = sp.S + 1;
    uint8_t* tr = image.data() + f.trans;
    auto dom = [&](int x, int y) { return x != 0 && y != 0 && sp.digraph[(x - 1) * sp.S + (y - 1)] == 1; };
    for (int act = 0; act < 3; ++act)
      for (int x = 0; x < s1; ++x)
        for (int y = 0; y < s1; ++y) {
          int nx = x, ny = y;
          if (x != y) {
            if (act == 0) {
              nx = y;
              ny = x;
            } else if (act == 1) {
              if (dom(x, y))
                ny = 0;
              else if (dom(y, x))
                nx = 0;
            } else {
              if (y == 0)
                ny = x;
              else if (x == 0)
                nx = y;
            }
          }
          tr[(x * s1 + y) * 4 + act] = (uint8_t)(nx | (ny << 4));
        }
    SlotDesc& sd = b->h_slots[i];
    std::memset(&sd, 0, sizeof sd);
    LatticeDesc& d = sd.d;
    d.lat = b->arena + f.lat;
    d.L = sp.L;
    d.pitch = escg_lattice_pitch(sp.L);
    d.P = p.P;
    d.GQ = p.GQ;
    d.cs = reinterpret_cast<int32_t*>(b->arena + f.tab);
    d.fs = d.cs + p.cs.size();
    d.fc = d.fs + p.fs.size();
    d.trans = b->arena + f.trans;
    d.key0 = (uint32_t)sp.seed;
    d.key1 = (uint32_t)(sp.seed >> 32);
    for (int r = 0; r < 10; ++r) {
      d.rk[2 * r] = d.key0 + (uint32_t)r * 0x9E3779B9u;
      d.rk[2 * r + 1] = d.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    const double I = sp.rates.interact, Pr = sp.rates.reproduce, X = sp.rates.exchange;
    const double R = (X + I) + Pr;
    const uint64_t tx = (uint64_t)std::floor(std::ldexp(X / R, 32) + 0.5);
    const uint64_t txi = (uint64_t)std::floor(std::ldexp((X + I) / R, 32) + 0.5);
    d.tx = tx >> 32 ? 0xFFFFFFFFu : (uint32_t)tx;
    d.txi = txi >> 32 ? 0xFFFFFFFFu : (uint32_t)txi;
    d.S = sp.S;
    d.uniform64 = 0;
    fill_perm24(d.perm24);
    sd.done = reinterpret_cast<uint32_t*>(b->arena + f.done);
    sd.max_mcs = (uint32_t)sp.max_mcs;
    sd.stop_at_extinction = sp.stop_at_extinction ? 1 : 0;
    sd.nb4 = p.P * p.P / 4;
  }
  std::vector<uint32_t> admit(n);
  for (int i = 0; i < n; ++i) admit[i] = (uint32_t)i;
  BatchCtl ctl{};
  ctl.n_admit = (uint32_t)n;
  e = cudaMemcpyAsync(b->arena, image.data(), total, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_slots, b->h_slots.data(), sizeof(SlotDesc) * n, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_states, 0, sizeof(SlotState) * n, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_admit, admit.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, b->stream);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    e = launch_init(b->h_slots[i].d, off[i].TE, b->stream);
    b->launches++;
  }
  if (e == cudaSuccess) {
    batch_count_kernel<<<n, 256, 0, b->stream>>>(b->d_slots, b->d_states, nullptr, n);
    e = cudaGetLastError();
    b->launches++;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // image is host stack memory
  if (e != cudaSuccess) {
    bset_err("batch initialisation failed: %s", cudaGetErrorString(e));
    free_batch(b);
    return nullptr;
  }
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<64>, 64, 0);
  b->grid[0] = sms * (per < 1 ? 1 : per);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<128>, 128, 0);
  b->grid[1] = sms * (per < 1 ? 1 : per);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<256>, 256, 0);
  b->grid[2] = sms * (per < 1 ? 1 : per);
  return b;
}

int escg_batch_run(escg_batch_t* b, uint64_t max_mcs) {
  if (!b) return ESCG_EINVAL;
  const uint32_t le = b->opt.log_every;
  uint64_t chunks_left = max_mcs ? (max_mcs + le - 1) / le : (b->mcs_budget_max + le - 1) / le + 1;
  // online autotuning of the CTA size: one chunk per candidate, timed with
  // events; the physical mapping never changes the results
  if (b->threads == 0) {
    const int cand[3] = {64, 128, 256};
    float best = 1e30f;
    int best_t = 256;
    for (int c = 0; c < 3 && chunks_left > 0; ++c) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, b->stream);
      if (enqueue_chunk(b, cand[c]) != cudaSuccess) {
        bset_err("batch chunk launch failed");
        return ESCG_ECUDA;
      }
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      --chunks_left;
      if (ms < best) {
        best = ms;
        best_t = cand[c];
      }
    }
    b->threads = best_t;
  }
  const int G = 16;   // chunks per graph replay
  if (b->opt.use_graph && !b->graph) {
    cudaGraph_t g;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      bset_err("CUDA graph capture failed to start");
      return ESCG_ECUDA;
    }
    for (int c = 0; c < G; ++c) {
      launch_compact(b);
      launch_batch_kernel(b, b->threads);
    }
    if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess ||
        cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) {
      bset_err("CUDA graph capture failed");
      return ESCG_ECUDA;
    }
    cudaGraphDestroy(g);
    b->graph_chunks = G;
  }
  while (chunks_left > 0) {
    if (b->graph && chunks_left >= (uint64_t)G) {
      if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) {
        bset_err("graph launch failed");
        return ESCG_ECUDA;
      }
      b->launches += 2 * G;
      chunks_left -= G;
    } else {
      if (enqueue_chunk(b, b->threads) != cudaSuccess) {
        bset_err("batch chunk launch failed");
        return ESCG_ECUDA;
      }
      chunks_left -= 1;
    }
    uint32_t n_active = 0;
    const int rc = active_count(b, &n_active);
    if (rc != ESCG_OK) return rc;
    if (n_active == 0) break;
  }
  // settle the MCS numbers and retirements of the last chunk
  if (launch_compact(b) != cudaSuccess) {
    bset_err("batch compaction launch failed");
    return ESCG_ECUDA;
  }
  b->launches++;
  return ESCG_OK;
}

int escg_batch_sync(escg_batch_t* b) {
  if (!b) return ESCG_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    bset_err("batch stream failed: %s", cudaGetErrorString(cudaGetLastError()));
    return ESCG_ECUDA;
  }
  BatchCtl ctl;
  if (cudaMemcpy(&ctl, b->d_ctl, sizeof ctl, cudaMemcpyDeviceToHost) != cudaSuccess) return ESCG_ECUDA;
  if (ctl.error & kErrTimeout) {
    bset_err("a bounded device-side wait timed out");
    return ESCG_ETIMEOUT;
  }
  return ESCG_OK;
}

int escg_batch_status(escg_batch_t* b, uint64_t* mcs_out, int32_t* extinct_out, uint64_t* counts16_out) {
  if (!b) return ESCG_EINVAL;
  int rc = escg_batch_sync(b);
  if (rc != ESCG_OK) return rc;
  std::vector<SlotState> st(b->n);
  if (cudaMemcpy(st.data(), b->d_states, sizeof(SlotState) * b->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ESCG_ECUDA;
  for (int i = 0; i < b->n; ++i) {
    if (mcs_out) mcs_out[i] = st[i].mcs;
    if (extinct_out) extinct_out[i] = (int32_t)st[i].stopped;
    if (counts16_out)
      for (int v = 0; v < kMaxStates; ++v) counts16_out[i * kMaxStates + v] = st[i].counts[v];
  }
  return ESCG_OK;
}

int32_t escg_batch_active(escg_batch_t* b) {
  if (!b) return -1;
  uint32_t n = 0;
  if (active_count(b, &n) != ESCG_OK) return -1;
  return (int32_t)n;
}

int escg_batch_snapshot(escg_batch_t* b, int32_t i, uint8_t* host_out) {
  if (!b || i < 0 || i >= b->n || !host_out) return ESCG_EINVAL;
  int rc = escg_batch_sync(b);
  if (rc != ESCG_OK) return rc;
  const LatticeDesc& d = b->h_slots[i].d;
  if (cudaMemcpy2D(host_out, d.L, d.lat, d.pitch, d.L, d.L, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ESCG_ECUDA;
  return ESCG_OK;
}

int32_t escg_batch_threads(escg_batch_t* b) { return b ? b->threads : 0; }
uint64_t escg_batch_launch_count(escg_batch_t* b) { return b ? b->launches : 0; }

void escg_batch_destroy(escg_batch_t* b) { free_batch(b); }

}  // extern "C"
