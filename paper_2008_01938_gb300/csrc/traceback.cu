// traceback.cu -- mcm_traceback: the optimal parenthesisation from the split
// table, on the device.
//
// The split table s defines a full binary tree over the chain: node (i, j),
// i < j, multiplies the product of matrices i..k by that of k+1..j, k =
// s[i][j] (Cormen et al., cited by the paper for the MCM recurrence).  The
// output lists the n-1 products in post-order, so every product comes after
// the two it consumes.  In post-order the products of the subtree (i, j)
// occupy j - i consecutive slots: its left subtree (i, k) the first k - i, its
// right subtree (k+1, j) the next j - k - 1, and (i, j) itself the last.  So
// each node knows its slot from its parent, and the tree is expanded one level
// per step: every node of a level reads its split, writes its product and
// appends its children to the next level, all in parallel.
#include <cuda_runtime.h>

#include <cstdint>

#include "api_internal.h"
#include "dp_common.cuh"

namespace {

struct Node {
  int32_t i, j, base;  // subtree (i, j), i < j; its products start at slot `base`
};

__global__ void __launch_bounds__(1024) traceback_kernel(const int16_t* __restrict__ s, int32_t n,
                                                         int32_t* __restrict__ steps, Node* front, Node* next,
                                                         int32_t* status) {
  __shared__ int32_t s_count[2];
  const int tid = threadIdx.x;
  if (tid == 0) {
    front[0] = Node{0, n - 1, 0};
    s_count[0] = 1;
    s_count[1] = 0;
  }
  __syncthreads();
  int cur = 0;
  // at most n - 1 levels (a chain-shaped tree); each level is one pass
  for (int level = 0; level < n; ++level) {
    const int cnt = s_count[cur];
    if (cnt == 0) break;
    for (int x = tid; x < cnt; x += blockDim.x) {
      const Node nd = front[x];
      const int k = s[(int64_t)nd.i * n + nd.j];
      if (k < nd.i || k >= nd.j) {  // not a split table of a solved chain
        dpk::set_status(status, DP_EINVAL);
        continue;
      }
      const int slot = nd.base + (nd.j - nd.i) - 1;
      steps[3 * slot + 0] = nd.i;
      steps[3 * slot + 1] = k;
      steps[3 * slot + 2] = nd.j;
      if (k > nd.i) next[atomicAdd(&s_count[cur ^ 1], 1)] = Node{nd.i, k, nd.base};
      if (k + 1 < nd.j) next[atomicAdd(&s_count[cur ^ 1], 1)] = Node{k + 1, nd.j, nd.base + (k - nd.i)};
    }
    __syncthreads();
    if (tid == 0) s_count[cur] = 0;
    Node* t = front;
    front = next;
    next = t;
    cur ^= 1;
    __syncthreads();
    if (*reinterpret_cast<volatile int32_t*>(status) != 0) break;
  }
}

}  // namespace

extern "C" dp_status mcm_traceback(const int16_t* s, int32_t n, int32_t* steps, int32_t* status_dev, void* stream) {
  if (n < 1 || n > 32767) return dph::fail(DP_EINVAL, "mcm_traceback: n = %d outside [1, 32767]", n);
  if (n == 1) return DP_OK;  // a single matrix: no products (steps may be NULL)
  if (!s || !steps) return dph::fail(DP_EINVAL, "mcm_traceback: NULL pointer argument");
  dph::DevState* ds = nullptr;
  dp_status rc = dph::current_dev(&ds);
  if (rc != DP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // two level buffers; a level holds at most n / 2 nodes (disjoint subtrees of >= 2 matrices)
  Node* buf = nullptr;
  const size_t per = (size_t)(n / 2 + 1) * sizeof(Node);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), 2 * per, st);
  if (e != cudaSuccess) return dph::fail_cuda(e, "mcm_traceback: level buffers");
  traceback_kernel<<<1, 1024, 0, st>>>(s, n, steps, buf, reinterpret_cast<Node*>(reinterpret_cast<uint8_t*>(buf) + per),
                                       status_dev ? status_dev : ds->status);
  e = cudaGetLastError();
  cudaError_t e2 = cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return dph::fail_cuda(e, "mcm_traceback: launch");
  if (e2 != cudaSuccess) return dph::fail_cuda(e2, "mcm_traceback: release");
  return DP_OK;
}
