// symbolize.cu -- label propagation (Sec. 5): each piece's symbol is the
// global id of its local group; no distance is evaluated again.
#include "kernels.cuh"

namespace jabba {

// One warp per domain: symbol[dom_piece_off[d] + j] =
// l2g[dom_group_off[d] + local_label[dom_slot_off[d] + j]].
__global__ void __launch_bounds__(256) k_symbolize(const int* local_label, const long long* dom_slot_off,
                                                   const int* dom_piece_cnt, const long long* dom_piece_off,
                                                   const long long* dom_group_off, long long n_domains,
                                                   const int* l2g, int* symbol) {
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long d = w; d < n_domains; d += nw) {
    const int n = dom_piece_cnt[d];
    const long long slot = dom_slot_off[d], po = dom_piece_off[d], go = dom_group_off[d];
    // four labels per lane, then their four gathers, in flight together
    for (int j0 = lane; j0 < n; j0 += 128) {
      int lab[4], s[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) lab[c] = j0 + 32 * c < n ? local_label[slot + j0 + 32 * c] : 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) s[c] = j0 + 32 * c < n ? l2g[go + lab[c]] : 0;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (j0 + 32 * c < n) symbol[po + j0 + 32 * c] = s[c];
    }
  }
}

void launch_symbolize(const int* local_label, const long long* dom_slot_off, const int* dom_piece_cnt,
                      const long long* dom_piece_off, const long long* dom_group_off, long long n_domains,
                      const int* l2g, int* symbol, Scratch& ws, cudaStream_t st) {
  if (n_domains <= 0) return;
  long long blocks = (n_domains + 7) / 8;
  if (blocks > (long long)ws.num_sms * 16) blocks = (long long)ws.num_sms * 16;
  k_symbolize<<<(unsigned)blocks, 256, 0, st>>>(local_label, dom_slot_off, dom_piece_cnt, dom_piece_off,
                                                 dom_group_off, n_domains, l2g, symbol);
}

}  // namespace jabba
