// Streaming stencil rows (stream.cu): inputs staged plane by plane in shared
// memory, each line of a thread's stencil footprint loaded once per plane.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace hhg {

// largest dynamic shared memory of a block (227 KB on sm_103a)
constexpr size_t kStreamMaxSmem = 232448;

// sets the shared-memory size attribute of every streaming kernel of one
// precision; call once before the first launch, outside stream capture
template <class T>
void stream_init();

// rows of op (OP_FULL, OP_BT or OP_BC) in MODE_SET / MODE_RES by the
// streaming kernels (one launch per pass): blocks of `threads` (64 / 128 /
// 256) threads of `sites` (FP32: 2 or 4; FP64: 4) consecutive sites each,
// owning sites x threads positions of the (i, j) plane and a run of k
// planes.  `tab` is the level's parameter image of op from
// stream_image<T>.  Returns false (nothing launched) if the combination is
// not supported, the level's pitch is not a multiple of four, the shared
// memory of a block would exceed kStreamMaxSmem, or a vector is not 16-byte
// aligned.
template <class T>
bool stream_rows(int disc, int varnu, int op, int mode, const Geo& g, const void* tab, const T* x, const T* b, T* y,
                 int threads, int sites, cudaStream_t s);

// the kernels of one translation unit: V = 2 or 4 sites per thread (FP64: 4)
template <class T, int V>
bool stream_rows_v(int disc, int varnu, int op, int mode, const Geo& g, const void* tab, const T* x, const T* b, T* y,
                   int threads, cudaStream_t s);
template <class T, int V>
void stream_init_v();
// the same passes as work items of the batch being recorded (batch.h; the
// batched translation units)
template <class T, int V>
bool stream_rows_record_v(int disc, int varnu, int op, int mode, const Geo& g, const void* tab, const T* x,
                          const T* b, T* y, int threads);

// the parameter image of op: weights w in the order of the FastTab images,
// and wc = 27 x NCB class sums of the boundary C stencil (class index
// ci + 3 cj + 9 ck, c = 0 low face, 1 inside, 2 high face; offsets in the
// order of stream_c_offsets); false if op has no streaming kernel
template <class T>
bool stream_image(int disc, int varnu, int op, const std::vector<double>& w, const std::vector<double>& wc,
                  std::vector<char>& out);

// the lattice offsets (di, dj, dk triples) of the boundary C stencil of op's
// pressure row (empty if it has no C terms)
bool stream_c_offsets(int disc, int varnu, int op, std::vector<int>& offsets);

}  // namespace hhg
