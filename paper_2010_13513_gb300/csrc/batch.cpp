// Recorder of a batch's kernel sequences and their merge into shared
// launches (declarations and the scheme in batch.h).
#include "batch.h"

#include <algorithm>

namespace hhg {

thread_local Recorder* g_rec = nullptr;

Recorder::~Recorder() {
  for (auto& kv : tables_) cudaFree(kv.second);
  if (items_dev_) cudaFree(items_dev_);
}

void Recorder::begin(int problem) {
  if (int(lists_.size()) <= problem) lists_.resize(problem + 1);
  cur_ = problem;
}

void Recorder::native(std::function<void(cudaStream_t)> f) {
  BatchOp op;
  op.native = std::move(f);
  lists_[cur_].push_back(std::move(op));
}

const void* Recorder::table(const void* host, size_t bytes) {
  const auto key = std::make_pair(host, bytes);
  auto it = tables_.find(key);
  if (it != tables_.end()) return it->second;
  void* d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess || cudaMemcpy(d, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    failed_ = true;
    if (d) cudaFree(d);
    return nullptr;
  }
  tables_[key] = d;
  return d;
}

namespace {
bool same_kind(const BatchOp& a, const BatchOp& b) {
  return !a.native && !b.native && a.fn == b.fn && a.block.x == b.block.x && a.block.y == b.block.y &&
         a.block.z == b.block.z && a.cluster == b.cluster;
}
}  // namespace

int Recorder::merge(std::vector<BatchLaunch>& out) {
  out.clear();
  if (failed_) return int(cudaErrorMemoryAllocation);
  const size_t np = lists_.size();
  std::vector<size_t> cur(np, 0);
  std::vector<unsigned char> host;
  std::vector<const BatchOp*> heads(np);
  for (;;) {
    // among the problems that are furthest behind (fewest ops taken), the
    // kind that most of them run next (ties: the earliest problem); every
    // problem whose next op is of that kind joins the launch
    size_t behind = ~size_t(0);
    for (size_t p = 0; p < np; ++p) {
      heads[p] = cur[p] < lists_[p].size() ? &lists_[p][cur[p]] : nullptr;
      if (heads[p]) behind = std::min(behind, cur[p]);
    }
    int best = -1, best_count = 0;
    for (size_t p = 0; p < np; ++p) {
      if (!heads[p] || cur[p] != behind) continue;
      int count = 1;
      if (!heads[p]->native)
        for (size_t q = p + 1; q < np; ++q)
          if (heads[q] && cur[q] == behind && same_kind(*heads[p], *heads[q])) ++count;
      if (count > best_count) {
        best = int(p);
        best_count = count;
      }
    }
    if (best < 0) break;
    const BatchOp& k = *heads[best];
    BatchLaunch l;
    if (k.native) {
      l.native = k.native;
      ++cur[best];
      out.push_back(std::move(l));
      continue;
    }
    l.fn = k.fn;
    l.block = k.block;
    l.cluster = k.cluster;
    l.items = (host.size() + 15) / 16 * 16;
    host.resize(l.items);
    int64_t blocks = 0;
    for (size_t p = 0; p < np; ++p) {
      if (!heads[p] || !same_kind(k, *heads[p])) continue;
      const BatchOp& op = *heads[p];
      const int64_t nb = int64_t(op.grid.x) * op.grid.y * op.grid.z;
      if (nb > 0) {
        BHead h{int(blocks), int(op.grid.x), int(op.grid.y), int(op.grid.z)};
        const size_t o = host.size();
        host.resize(o + op.item_size, 0);
        std::memcpy(host.data() + o, &h, sizeof(h));
        std::memcpy(host.data() + o + op.args_off, op.args.data(), op.args.size());
        blocks += nb;
        ++l.n;
        l.smem = std::max(l.smem, op.smem);
      }
      ++cur[p];
    }
    if (blocks >= (int64_t(1) << 31)) return int(cudaErrorInvalidConfiguration);
    l.blocks = int(blocks);
    if (l.n > 0) out.push_back(std::move(l));
  }
  if (items_dev_) {
    cudaFree(items_dev_);
    items_dev_ = nullptr;
  }
  if (!host.empty()) {
    cudaError_t e = cudaMalloc(&items_dev_, host.size());
    if (e == cudaSuccess) e = cudaMemcpy(items_dev_, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return int(e);
  }
  return 0;
}

cudaError_t launch_merged(const BatchLaunch& l, const unsigned char* items, cudaStream_t s) {
  if (l.native) {
    l.native(s);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(l.blocks), 1, 1);
  cfg.blockDim = l.block;
  cfg.dynamicSmemBytes = l.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (l.cluster > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(l.cluster);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  const void* p = items + l.items;
  int n = l.n;
  void* args[] = {&p, &n};
  return cudaLaunchKernelExC(&cfg, l.fn, args);
}

}  // namespace hhg
