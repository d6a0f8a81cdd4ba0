// Swap counts (Appendix "Swaps performed by Curveball and Global Curveball"):
// a trade performs as many neighbourhood swaps as edge ends that change node
// (twice the pairs of neighbours it exchanges), out of deg(u) + deg(v)
// possible.  With the "swap_stats" option on, every global super step adds
// its counts: the entries whose side word marks a move to the other node of
// their trade (the untraded node of an odd n never moves), and the degrees
// of the traded positions.  Uniform trades add theirs in the executor
// (uniform.cu).
#include "cb_internal.cuh"

namespace cb {
namespace {

// out[0] += moved entries among all nnz (bit 0 of each side word), out[1] += rp[two_t] (the entries of
// the traded positions' rows in the step just done).
__global__ void k_count_flips(const uint16_t* __restrict__ stash, int64_t nnz, const int64_t* __restrict__ rp,
                              int64_t two_t, unsigned long long* out) {
  const int64_t end = nnz;
  const int64_t words = end >> 1;
  const int64_t tid = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  unsigned long long local = 0;
  const uint32_t* w = reinterpret_cast<const uint32_t*>(stash);
  for (int64_t i = tid; i < words; i += stride) local += __popc(__ldg(w + i) & 0x00010001u);
  for (int64_t e = (words << 1) + tid; e < end; e += stride) local += stash[e] & 1u;
#pragma unroll
  for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(&out[0], local);
  if (tid == 0) atomicAdd(&out[1], static_cast<unsigned long long>(rp[two_t]));
}

}  // namespace

int count_swaps(Graph* h) {
  if (!h->swaps || h->n < 2) return CB_OK;
  // the step just done read the rows of the other ping-pong side
  const int64_t two_t = 2 * (h->n / 2);
  const unsigned grid = static_cast<unsigned>(h->num_sms * 4);
  k_count_flips<<<grid, 256, 0, h->stream>>>(h->stash, h->nnz, h->rp[1 - h->cur], two_t,
                                             reinterpret_cast<unsigned long long*>(h->swaps));
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  return CB_OK;
}

int set_swap_stats(Graph* h, bool on) {
  if (on && h->nseg != 1) return fail(h, CB_EINVAL, "swap counts are for handles of one graph");
  h->swap_stats = on;
  if (!on) return CB_OK;
  if (!h->swaps) {
    void* p = nullptr;
    if (dev_alloc(h, &p, 2 * sizeof(int64_t))) return fail(h, CB_ENOMEM, "device allocation failed");
    h->swaps = static_cast<int64_t*>(p);
  }
  CB_CUDA(h, cudaMemsetAsync(h->swaps, 0, 2 * sizeof(int64_t), h->stream));
  return CB_OK;
}

}  // namespace cb

extern "C" int cb_swap_counts(cb_handle h, int64_t* performed, int64_t* possible) {
  using namespace cb;
  if (!h || !performed || !possible) return fail(h, CB_EINVAL, "bad argument");
  int64_t v[2] = {0, 0};
  if (h->swaps) {
    CB_CUDA(h, cudaMemcpyAsync(v, h->swaps, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    CB_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  *performed = v[0];
  *possible = v[1];
  return CB_OK;
}
