// concat.cu — streams of consecutive shards of one field joined into the
// field's stream (Sec. VI-B5: every node compresses its part and the
// compressed data are gathered at a root).
//
// Blocks are independent (Sec. IV-A), so when every shard but the last holds
// whole blocks, the field's stream is the shards' sections laid end to end:
// rates, outliers, sign words and plane words (Fig. 3), each section at the
// running totals of the shards before it, with one new header. A plan kernel
// (one CTA) reads the shards' headers, checks that they form one field,
// writes the prefixes into the shard table and the output's header and
// padding; a copy kernel then moves every section with a grid-stride loop per
// shard. Nothing is decoded.
#include <vector>

#include "hz_kernels.cuh"

namespace hz {

// Shard table in the workspace: the host writes c and bytes; the plan kernel
// fills in the rest.
struct ShardRec {
  const uint8_t* c;
  uint64_t bytes;
  uint64_t nb, nnc, R, o_out, o_sign, o_plane;
  uint64_t pnb, pnnc, pR;  // blocks, non-constant blocks and plane words before the shard
};
struct ConcatPlan {
  uint64_t ok, NB, NNC, R;
};

constexpr int CC_PLAN_THREADS = 256;

// One CTA. Thread t takes a contiguous run of shards: it parses their headers
// (filling the table), sums their blocks, words and values, and notes the
// first shard that breaks a rule; a scan over the threads then gives every
// shard its prefixes, and thread 0 writes the header, the padding and the size.
__global__ void __launch_bounds__(CC_PLAN_THREADS) k_concat_plan(
    ShardRec* rec, uint32_t k, uint32_t d0, uint32_t d1, uint32_t d2, uint32_t ndims,
    uint8_t* out, uint64_t cap, uint64_t* out_bytes, Ws ws) {
  __shared__ unsigned long long s_sum[4][CC_PLAN_THREADS];
  __shared__ unsigned int s_qb[CC_PLAN_THREADS];
  __shared__ unsigned long long s_bad[CC_PLAN_THREADS];  // (first bad shard << 8) | code
  ConcatPlan* plan = reinterpret_cast<ConcatPlan*>(rec + k);
  const int tid = threadIdx.x;
  const uint32_t per = (k + CC_PLAN_THREADS - 1) / CC_PLAN_THREADS;
  const uint32_t s0 = min(k, (uint32_t)tid * per), s1 = min(k, s0 + per);
  const Info h0 = parse_header(rec[0].c, rec[0].bytes);
  unsigned long long nb = 0, nnc = 0, R = 0, n = 0, badw = ~0ull;
  uint32_t qb = 0;
  for (uint32_t s = s0; s < s1; s++) {
    const Info h = parse_header(rec[s].c, rec[s].bytes);
    int code = 0;
    if (!h.ok) code = HOSZP_ERR_FORMAT;
    else if (__float_as_uint(h.eps_q) != __float_as_uint(h0.eps_q) ||
             __double_as_longlong(h.eps) != __double_as_longlong(h0.eps) ||
             (s + 1 < k && h.n % L != 0))
      code = HOSZP_ERR_MISMATCH;
    if (code) {
      if (badw == ~0ull) badw = ((unsigned long long)s << 8) | (unsigned)(-code);
      continue;
    }
    rec[s].nb = h.nb;
    rec[s].nnc = h.nnc;
    rec[s].R = h.R;
    rec[s].o_out = h.o_out;
    rec[s].o_sign = h.o_sign;
    rec[s].o_plane = h.o_plane;
    rec[s].pnb = nb;  // within the thread's run; the run's base is added below
    rec[s].pnnc = nnc;
    rec[s].pR = R;
    nb += h.nb;
    nnc += h.nnc;
    R += h.R;
    n += h.n;
    qb = max(qb, h.qbound);
  }
  s_sum[0][tid] = nb;
  s_sum[1][tid] = nnc;
  s_sum[2][tid] = R;
  s_sum[3][tid] = n;
  s_qb[tid] = qb;
  s_bad[tid] = badw;
  __syncthreads();
  if (tid == 0) {  // exclusive prefixes of the runs, totals, first error
    unsigned long long a[4] = {0, 0, 0, 0}, fb = ~0ull;
    uint32_t q = 0;
    for (int t = 0; t < CC_PLAN_THREADS; t++) {
      for (int j = 0; j < 4; j++) {
        const unsigned long long v = s_sum[j][t];
        s_sum[j][t] = a[j];
        a[j] += v;
      }
      q = max(q, s_qb[t]);
      fb = min(fb, s_bad[t]);
    }
    int bad = fb != ~0ull ? -(int)(fb & 0xffu) : 0;
    const uint64_t prod = (uint64_t)d0 * (ndims > 1 ? d1 : 1u) * (ndims > 2 ? d2 : 1u);
    if (!bad && prod != a[3]) bad = HOSZP_ERR_ARG;
    const uint64_t NB = a[0], NNC = a[1], RT = a[2];
    const uint64_t size = bad ? 0 : stream_bytes(NB, NNC, RT);
    if (!bad && size > cap) bad = HOSZP_ERR_CAPACITY;
    plan->ok = bad ? 0 : 1;
    plan->NB = NB;
    plan->NNC = NNC;
    plan->R = RT;
    if (bad) {
      set_status(ws.status, bad);
      *out_bytes = 0;
    } else {
      hoszp_header H;
      H.magic = HOSZP_MAGIC;
      H.version = HOSZP_VERSION;
      H.dtype = 0;
      H.ndims = (uint8_t)ndims;
      H.dims[0] = d0;
      H.dims[1] = ndims > 1 ? d1 : 0u;
      H.dims[2] = ndims > 2 ? d2 : 0u;
      H.eps_q = h0.eps_q;
      H.n = a[3];
      H.eps = h0.eps;
      H.nnc = NNC;
      H.R = RT;
      H.qbound = q;
      H.block = HOSZP_BLOCK;
      *reinterpret_cast<hoszp_header*>(out) = H;
      // zero padding after the rate and outlier sections and at the stream's end
      for (uint64_t b = HOSZP_HEADER_BYTES + NB; b < off_outlier(NB); b++) out[b] = 0;
      for (uint64_t b = off_outlier(NB) + 4 * NB; b < off_sign(NB); b++) out[b] = 0;
      for (uint64_t b = off_plane(NB, NNC) + 8 * RT; b < size; b++) out[b] = 0;
      *out_bytes = size;
    }
  }
  __syncthreads();
  for (uint32_t s = s0; s < s1; s++) {  // the run's base
    rec[s].pnb += s_sum[0][tid];
    rec[s].pnnc += s_sum[1][tid];
    rec[s].pR += s_sum[2][tid];
  }
}

__global__ void __launch_bounds__(256) k_concat_copy(const ShardRec* rec, uint32_t k,
                                                     uint8_t* __restrict__ out) {
  const ConcatPlan plan = *reinterpret_cast<const ConcatPlan*>(rec + k);
  if (!plan.ok) return;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint8_t* const orate = out + HOSZP_HEADER_BYTES;
  int* const oout = reinterpret_cast<int*>(out + off_outlier(plan.NB));
  uint64_t* const osign = reinterpret_cast<uint64_t*>(out + off_sign(plan.NB));
  uint64_t* const oplane = reinterpret_cast<uint64_t*>(out + off_plane(plan.NB, plan.NNC));
  for (uint32_t s = 0; s < k; s++) {
    const ShardRec r = rec[s];
    const uint8_t* c = r.c;
    for (uint64_t i = i0; i < r.nb; i += stride) orate[r.pnb + i] = c[HOSZP_HEADER_BYTES + i];
    const int* cout = reinterpret_cast<const int*>(c + r.o_out);
    for (uint64_t i = i0; i < r.nb; i += stride) oout[r.pnb + i] = __ldg(cout + i);
    const uint64_t* csign = reinterpret_cast<const uint64_t*>(c + r.o_sign);
    for (uint64_t i = i0; i < r.nnc; i += stride) osign[r.pnnc + i] = __ldg(csign + i);
    const uint64_t* cplane = reinterpret_cast<const uint64_t*>(c + r.o_plane);
    for (uint64_t i = i0; i < r.R; i += stride) oplane[r.pR + i] = __ldg(cplane + i);
  }
}

// Words of workspace staging the table of k shards needs.
uint64_t concat_table_words(uint32_t k) {
  return ((uint64_t)k * sizeof(ShardRec) + sizeof(ConcatPlan) + 7) / 8;
}

cudaError_t launch_concat(const Launch& lc, uint32_t k, const void* const* streams,
                          const size_t* bytes, const uint32_t dims[3], uint32_t ndims,
                          uint8_t* out, uint64_t cap, uint64_t* out_bytes, Ws ws) {
  ShardRec* rec = reinterpret_cast<ShardRec*>(ws.staging);
  std::vector<ShardRec> host(k);
  for (uint32_t s = 0; s < k; s++) {
    host[s] = ShardRec{};
    host[s].c = static_cast<const uint8_t*>(streams[s]);
    host[s].bytes = bytes[s];
  }
  // pageable source: the call returns once the table is staged for the copy
  cudaError_t e = cudaMemcpyAsync(rec, host.data(), sizeof(ShardRec) * k, cudaMemcpyHostToDevice,
                                  lc.stream);
  if (e != cudaSuccess) return e;
  k_concat_plan<<<1, CC_PLAN_THREADS, 0, lc.stream>>>(rec, k, dims[0], dims[1], dims[2], ndims, out, cap,
                                        out_bytes, ws);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_concat_copy<<<lc.grid * 4, 256, 0, lc.stream>>>(rec, k, out);
  return cudaGetLastError();
}

}  // namespace hz
