// Merged launches of a batch of independent problems.
//
// A batch solve first records the kernel sequence of every problem's FMG
// instead of launching it: each launch becomes an op (the batched variant of
// its kernel, its grid and block, and its arguments as plain bytes).  The
// recorder then walks the problems' sequences side by side and merges the
// next ops of all problems that run the same kernel with the same block
// shape into ONE launch over the flat list of (problem op, block) work
// items; problems never share data, so any interleaving that keeps each
// problem's own order is exact.  A merged launch takes the concatenated
// grids of its items along x; block b finds its item (the last item whose
// first block is <= b) and its local block index within the item's own
// (gx, gy, gz) grid, and runs the same device code as the plain kernel with
// that item's arguments.  Launch sites without a batched variant are
// recorded as "native" ops and replayed unmerged.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <type_traits>
#include <utility>
#include <vector>

namespace hhg {

struct BHead {
  int start;           // first block of the item in the merged grid
  int gx, gy, gz;      // the item's own grid
};

template <class A>
struct BItem {
  BHead h;
  A a;
};

#ifdef __CUDACC__
// the item of merged block blockIdx.x and the block's index within it
template <class A>
__device__ __forceinline__ const BItem<A>& batch_item(const void* items, int n, uint3& bid, uint3& gdim) {
  const BItem<A>* it = static_cast<const BItem<A>*>(items);
  const int b = int(blockIdx.x);
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (it[mid].h.start <= b) lo = mid;
    else hi = mid - 1;
  }
  const BItem<A>& r = it[lo];
  const unsigned l = unsigned(b - r.h.start), gx = unsigned(r.h.gx), gy = unsigned(r.h.gy);
  bid = make_uint3(l % gx, (l / gx) % gy, l / (gx * gy));
  gdim = make_uint3(gx, gy, unsigned(r.h.gz));
  return r;
}
#endif

// One recorded op: a batched kernel with its arguments, or a native launch.
struct BatchOp {
  const void* fn = nullptr;              // batched kernel: void(const void* items, int n)
  dim3 grid, block;
  size_t smem = 0;
  int cluster = 1;
  int kernels = 1;                       // kernel launches the op stands for (0: a memset)
  size_t item_size = 0, args_off = 0;
  std::vector<unsigned char> args;
  std::function<void(cudaStream_t)> native;
};

// A merged launch of the batch graph.
struct BatchLaunch {
  const void* fn = nullptr;
  dim3 block;
  int blocks = 0, cluster = 1, n = 0;
  size_t smem = 0, items = 0;            // byte offset of the items in the item buffer
  std::function<void(cudaStream_t)> native;
};

class Recorder {
 public:
  ~Recorder();
  void begin(int problem);               // ops recorded next belong to this problem
  template <class A>
  void add(const void* fn, dim3 grid, dim3 block, size_t smem, int cluster, const A& a, int kernels = 1) {
    static_assert(std::is_trivially_copyable<A>::value, "batched arguments are copied as bytes");
    BatchOp op;
    op.fn = fn;
    op.grid = grid;
    op.block = block;
    op.smem = smem;
    op.cluster = cluster;
    op.kernels = kernels;
    op.item_size = sizeof(BItem<A>);
    op.args_off = offsetof(BItem<A>, a);
    op.args.resize(sizeof(A));
    std::memcpy(op.args.data(), &a, sizeof(A));
    lists_[cur_].push_back(std::move(op));
  }
  void native(std::function<void(cudaStream_t)> f);
  // device copy of a host table (kept until the recorder is destroyed; one
  // copy per host address and size)
  const void* table(const void* host, size_t bytes);
  // merges the recorded sequences; uploads the items; returns 0 or a CUDA error
  int merge(std::vector<BatchLaunch>& out);
  const unsigned char* items() const { return items_dev_; }
  // kernel launches of the recorded batched ops (the native ops count when replayed)
  int64_t batched_kernels() const {
    int64_t n = 0;
    for (const auto& l : lists_)
      for (const BatchOp& op : l) n += op.native ? 0 : op.kernels;
    return n;
  }
  bool failed() const { return failed_; }

 private:
  std::vector<std::vector<BatchOp>> lists_;
  int cur_ = 0;
  std::map<std::pair<const void*, size_t>, void*> tables_;
  unsigned char* items_dev_ = nullptr;
  bool failed_ = false;
};

// set while a batch records its problems' kernel sequences (else null)
extern thread_local Recorder* g_rec;

// launches one merged op on s (items at items + l.items)
cudaError_t launch_merged(const BatchLaunch& l, const unsigned char* items, cudaStream_t s);

}  // namespace hhg
