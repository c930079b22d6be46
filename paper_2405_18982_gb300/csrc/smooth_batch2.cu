// Ragged batch of independent 2D problems: one persistent launch per
// smoothing stage of the V-cycle across all members (the register-direct 2D
// colour-pass body of smooth_int2.cuh, with coherent loads of x).
//
// The members of a batch have different degrees and sizes, but every member's
// level l has N = 2^(l+1) cells per direction (coarsest level 2 x 2), so the
// V-cycles of all members line up level by level.  A stage "smoothing step on
// level l" of the whole batch is one cooperative launch: a work list of
// (member, patch chunk) items per colour -- interior and domain-boundary
// patch chunks of every member that has level l -- walked by all CTAs, the
// four colours (2D; reversed in post-smoothing) separated by bounded grid
// barriers.  Each item dispatches on its member's degree to the compile-time
// colour-pass body of that degree (Algorithm 1 with the fast-diagonalisation
// local solve of Eq. inverse2d), reading that member's 1D operators from
// device memory.  Members are independent, so one barrier for all members
// only makes a member wait for others; a member's colour c + 1 still starts
// after its colour c.
#include <array>
#include <cstring>
#include <vector>

#include "smoother_impl.cuh"

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchNNmin = 3, kBatchNNmax = 7;  // degrees 2..6

// one chunk = the patches one CTA of the register-direct 2D colour pass
// handles (I2<NN>::PPC of them, TPP threads each, at most 256 threads)
template <int NN, bool BND>
constexpr int b2_ppc() {
  return I2<NN, float, BND>::PPC;
}
constexpr int b2_max(int a, int b) { return a > b ? a : b; }
template <int NN>
constexpr int b2_bytes_nn() {
  return b2_max((int)I2<NN, float, false>::SMEM, (int)I2<NN, float, true>::SMEM);
}
constexpr int kBatchSmem =
    b2_max(b2_max(b2_max(b2_bytes_nn<3>(), b2_bytes_nn<4>()), b2_max(b2_bytes_nn<5>(), b2_bytes_nn<6>())),
           b2_bytes_nn<7>());
static_assert(I2<3, float, false>::THREADS <= kBatchThreads && I2<3, float, true>::THREADS <= kBatchThreads &&
                  I2<7, float, false>::THREADS <= kBatchThreads && I2<7, float, true>::THREADS <= kBatchThreads,
              "chunk larger than the batched CTA");

// One member on one level: its vectors, its operator sets (device), its
// patch grids per colour and the first work item of each colour.
struct B2Member {
  const float* b;
  float* x;
  const void* ops_i;  // SmoothOps of the interior patches (register-direct 2D layout)
  const void* ops_b;  // SmoothOps of the four domain-boundary patch types
  PatchGrid g[4];
  long long first[4];
  const int* active;  // the member's Krylov "active" flag (device): 0 once it has converged
  int nn, N, consistent, pad_;
};

template <int NN>
__device__ __forceinline__ void b2_item(const B2Member& m, int colour, long long local, unsigned char* sm) {
  using CI = I2<NN, float, false>;
  using CB = I2<NN, float, true>;
  constexpr int PI = CI::PPC, PB = CB::PPC;
  const PatchGrid& g = m.g[colour];
  const long long chi = (g.n_int + PI - 1) / PI;
  if (local < chi) {
    const auto& ops = *reinterpret_cast<const SmoothOps<CI::PO, CI::P, float, CI::NT>*>(m.ops_i);
    int2_body<NN, float, false, false>(ops, sm, local * PI, colour, m.b, m.x, m.N, m.consistent, g);
  } else {
    const auto& ops = *reinterpret_cast<const SmoothOps<CB::PO, CB::P, float, CB::NT>*>(m.ops_b);
    int2_body<NN, float, true, false>(ops, sm, (local - chi) * PB, colour, m.b, m.x, m.N, m.consistent, g);
  }
}

__global__ void __launch_bounds__(kBatchThreads, 2)
    batch_step2_kernel(const B2Member* __restrict__ mem, int nmem, int reverse, long long t0, long long t1,
                       long long t2, long long t3, unsigned int* bar, int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  const long long tot[4] = {t0, t1, t2, t3};
  for (int ci = 0; ci < 4; ++ci) {
    const int c = reverse ? 3 - ci : ci;
    for (long long q = blockIdx.x; q < tot[c]; q += gridDim.x) {
      // the member owning item q: the last one whose first item is <= q
      int lo = 0, hi = nmem - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mem[mid].first[c] <= q) lo = mid;
        else hi = mid - 1;
      }
      const B2Member& m = mem[lo];
      // a converged member's V-cycle output is not used: skip its patches
      // (one thread reads the flag, so the decision is uniform in the CTA)
      __shared__ int s_skip;
      if (threadIdx.x == 0) s_skip = (m.active && *(volatile const int*)m.active == 0) ? 1 : 0;
      __syncthreads();
      const bool skip = s_skip != 0;
      __syncthreads();
      if (skip) continue;
      const long long local = q - m.first[c];
      switch (m.nn) {
        case 3: b2_item<3>(m, c, local, sm); break;
        case 4: b2_item<4>(m, c, local, sm); break;
        case 5: b2_item<5>(m, c, local, sm); break;
        case 6: b2_item<6>(m, c, local, sm); break;
        default: b2_item<7>(m, c, local, sm); break;
      }
      __syncthreads();  // the next item re-lays out the prefix and the slots
    }
    if (ci + 1 < 4 && !grid_barrier(bar, status, gridDim.x)) return;
  }
}

template <int NN>
long long b2_chunks(const PatchGrid& g) {
  constexpr int PI = b2_ppc<NN, false>(), PB = b2_ppc<NN, true>();
  return (g.n_int + PI - 1) / PI + (g.n_bnd + PB - 1) / PB;
}

long long b2_chunks_nn(int nn, const PatchGrid& g) {
  switch (nn) {
    case 3: return b2_chunks<3>(g);
    case 4: return b2_chunks<4>(g);
    case 5: return b2_chunks<5>(g);
    case 6: return b2_chunks<6>(g);
    default: return b2_chunks<7>(g);
  }
}

template <int NN>
size_t b2_ops_i_bytes() {
  using CI = I2<NN, float, false>;
  return sizeof(SmoothOps<CI::PO, CI::P, float, CI::NT>);
}
template <int NN>
size_t b2_ops_bytes() {
  using CB = I2<NN, float, true>;
  return b2_ops_i_bytes<NN>() + sizeof(SmoothOps<CB::PO, CB::P, float, CB::NT>);
}
// bytes of a member's two operator sets (all = true) or of the interior one
size_t b2_ops_bytes_nn(int nn, bool all = true) {
  switch (nn) {
    case 3: return all ? b2_ops_bytes<3>() : b2_ops_i_bytes<3>();
    case 4: return all ? b2_ops_bytes<4>() : b2_ops_i_bytes<4>();
    case 5: return all ? b2_ops_bytes<5>() : b2_ops_i_bytes<5>();
    case 6: return all ? b2_ops_bytes<6>() : b2_ops_i_bytes<6>();
    default: return all ? b2_ops_bytes<7>() : b2_ops_i_bytes<7>();
  }
}

// host: the member's two operator sets of `level` into `dst` (interior, then
// boundary)
template <int NN>
void b2_fill_ops(const sipg_handle* h, int level, unsigned char* dst) {
  using CI = I2<NN, float, false>;
  using CB = I2<NN, float, true>;
  SmoothOps<CI::PO, CI::P, float, CI::NT> oi;
  make_ops<CI::PO, CI::P, false, float>(h->hcst<float>(level), 0, oi.t[0]);
  SmoothOps<CB::PO, CB::P, float, CB::NT> ob;
  for (int t = 0; t < CB::NT; ++t) make_ops<CB::PO, CB::P, true, float>(h->hcst<float>(level), t, ob.t[t]);
  memcpy(dst, &oi, sizeof(oi));
  memcpy(dst + sizeof(oi), &ob, sizeof(ob));
}
void b2_fill_ops_nn(int nn, const sipg_handle* h, int level, unsigned char* dst) {
  switch (nn) {
    case 3: b2_fill_ops<3>(h, level, dst); break;
    case 4: b2_fill_ops<4>(h, level, dst); break;
    case 5: b2_fill_ops<5>(h, level, dst); break;
    case 6: b2_fill_ops<6>(h, level, dst); break;
    default: b2_fill_ops<7>(h, level, dst); break;
  }
}

size_t align256b(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// A plan: per level, the member table and the item counts per colour, in
// caller-owned device memory; plus the grid-barrier word of the batched
// launches.
struct BatchPlan2 {
  std::vector<const B2Member*> table;           // per level (device), null if no member has it
  std::vector<int> count;                       // members per level
  std::vector<std::array<long long, 4>> total;  // items per level and colour
  unsigned int* bar = nullptr;                  // device: [count, generation, status]
  int grid = 0;                                 // cooperative grid
};

bool batch2_supported(const std::vector<sipg_handle*>& hs) {
  if (hs.empty()) return false;
  for (const sipg_handle* h : hs) {
    if (h->prm.dim != 2 || h->prm.vcycle_precision != SIPG_FP32 || h->prm.nrhs != 1) return false;
    if (h->prm.smoother != SIPG_SMOOTHER_CONSISTENT && h->prm.smoother != SIPG_SMOOTHER_PAPER) return false;
    if (h->n < kBatchNNmin || h->n > kBatchNNmax) return false;
    if (h->lv[0].N != 2) return false;  // levels line up only from a 2 x 2 coarsest level
  }
  return true;
}

size_t batch2_plan_bytes(const std::vector<sipg_handle*>& hs) {
  size_t total = 256;  // barrier words
  for (const sipg_handle* h : hs)
    for (int l = 1; l <= h->L; ++l) total += align256b(b2_ops_bytes_nn(h->n));
  int levels = 0;
  for (const sipg_handle* h : hs) levels = std::max(levels, h->L + 1);
  total += (size_t)levels * align256b(sizeof(B2Member) * hs.size());
  return total;
}

// Builds the plan in `dev` (batch2_plan_bytes bytes, 256-aligned, caller
// owned): the operator sets and member tables are written on the host and
// copied (synchronously: bind time).  The member vectors are each handle's
// level vectors (the FP32 V-cycle buffers on the finest level).
cudaError_t batch2_plan_build(const std::vector<sipg_handle*>& hs, char* dev, BatchPlan2** out) {
  *out = nullptr;
  int levels = 0;
  for (const sipg_handle* h : hs) levels = std::max(levels, h->L + 1);
  std::vector<unsigned char> host(batch2_plan_bytes(hs), 0);
  size_t off = 256;
  // operator sets
  std::vector<std::vector<size_t>> ops_off(hs.size());
  for (size_t i = 0; i < hs.size(); ++i) {
    ops_off[i].assign(hs[i]->L + 1, 0);
    for (int l = 1; l <= hs[i]->L; ++l) {
      b2_fill_ops_nn(hs[i]->n, hs[i], l, host.data() + off);
      ops_off[i][l] = off;
      off += align256b(b2_ops_bytes_nn(hs[i]->n));
    }
  }
  BatchPlan2* p = new BatchPlan2();
  p->table.assign(levels, nullptr);
  p->count.assign(levels, 0);
  p->total.assign(levels, {0, 0, 0, 0});
  for (int l = 1; l < levels; ++l) {
    std::vector<B2Member> tab;
    std::array<long long, 4> run = {0, 0, 0, 0};
    for (size_t i = 0; i < hs.size(); ++i) {
      const sipg_handle* h = hs[i];
      if (l > h->L) continue;
      B2Member m{};
      const bool finest = l == h->L;
      m.b = finest ? reinterpret_cast<const float*>(h->ws + h->off_bL) : reinterpret_cast<const float*>(h->vb(l));
      m.x = finest ? reinterpret_cast<float*>(h->ws + h->off_xL) : reinterpret_cast<float*>(h->vx(l));
      const size_t oi = ops_off[i][l];
      m.nn = h->n;
      m.N = h->lv[l].N;
      m.consistent = h->prm.smoother == SIPG_SMOOTHER_CONSISTENT ? 1 : 0;
      m.active = &h->scalars()->active;
      m.ops_i = dev + oi;                                   // interior set, then the boundary sets
      m.ops_b = dev + oi + b2_ops_bytes_nn(h->n, false);
      for (int c = 0; c < 4; ++c) {
        m.g[c] = make_grid(2, m.N, c);
        m.first[c] = run[c];
        run[c] += b2_chunks_nn(m.nn, m.g[c]);
      }
      tab.push_back(m);
    }
    p->count[l] = (int)tab.size();
    p->total[l] = run;
    if (tab.empty()) continue;
    memcpy(host.data() + off, tab.data(), sizeof(B2Member) * tab.size());
    p->table[l] = reinterpret_cast<const B2Member*>(dev + off);
    off += align256b(sizeof(B2Member) * hs.size());
  }
  p->bar = reinterpret_cast<unsigned int*>(dev);
  cudaError_t e = cudaMemcpy(dev, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete p;
    return e;
  }
  int per_sm = 0;
  e = smem_opt_in_occupancy(reinterpret_cast<const void*>(batch_step2_kernel), kBatchThreads, kBatchSmem, &per_sm);
  if (e != cudaSuccess) {
    delete p;
    return e;
  }
  int dev_id = 0, sms = 0;
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
  p->grid = per_sm * sms;
  if (p->grid <= 0) {
    delete p;
    return cudaErrorNotSupported;
  }
  *out = p;
  return cudaSuccess;
}

void batch2_plan_free(BatchPlan2* p) { delete p; }

int batch2_levels(const BatchPlan2* p) { return (int)p->table.size(); }

// One smoothing step (reverse = post-smoothing order) on level l of every
// member that has it: one cooperative launch.
cudaError_t batch2_step(const BatchPlan2* p, int level, int reverse, cudaStream_t s) {
  if (level <= 0 || level >= (int)p->table.size() || !p->table[level]) return cudaSuccess;
  const auto& t = p->total[level];
  const long long most = std::max(std::max(t[0], t[1]), std::max(t[2], t[3]));
  const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(p->grid, most));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBatchThreads);
  cfg.dynamicSmemBytes = kBatchSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_step2_kernel, p->table[level], p->count[level], reverse, t[0], t[1], t[2],
                            t[3], p->bar, reinterpret_cast<int*>(p->bar + 2));
}

// the bounded grid barrier's status word of the batched launches (0: fine)
int* batch2_status(const BatchPlan2* p) { return reinterpret_cast<int*>(p->bar + 2); }
