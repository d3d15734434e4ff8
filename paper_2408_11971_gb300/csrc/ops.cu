// ops.cu — homomorphic operators on compressed streams (Sec. V, Table 2):
//   negation and scalar addition in fully compressed space (workflow 1),
//   scalar multiplication through the quantized integers (workflow 3),
//   element-wise addition through the decoded deltas (workflow 2).
#include "hz_decode.cuh"
#include "hz_kernels.cuh"

namespace hz {

// ---------------------------------------------------------------- scalar quantization
// Eq. 3 for a scalar operand s (a double), evaluated exactly with 128-bit
// integers: with s = ms 2^es and e = me 2^ee (me, ms integers),
// (s + e) / (2e) = (ms 2^(es-ee) + me) / (2 me), and the floor of that ratio
// is an integer division rounded toward minus infinity. Returns false when
// |rho| would exceed HOSZP_QLIM.
__device__ bool quantize_scalar(double s, float e, long long& rho) {
  const double de = (double)e;
  if (fabs(s) < de) {
    rho = 0;
    return true;
  }
  if (fabs(s) / de > 2.0 * (double)HOSZP_QLIM + 4.0) return false;
  int es, ee;
  const double fs = frexp(s, &es), fe = frexp(de, &ee);
  const long long ms = (long long)ldexp(fs, 53), me = (long long)ldexp(fe, 53);
  es -= 53;
  ee -= 53;
  const int sh = es - ee;  // |s|/e in [1, 2^32) => sh in [-1, 33]
  __int128 num, den;
  if (sh >= 0) {
    num = (__int128)ms * ((__int128)1 << sh) + me;
    den = (__int128)me * 2;
  } else {
    num = (__int128)ms + (__int128)me * ((__int128)1 << (-sh));
    den = (__int128)me * ((__int128)1 << (1 - sh));
  }
  __int128 qq = num / den;
  if (num % den != 0 && num < 0) qq -= 1;
  if (qq > HOSZP_QLIM || qq < -(__int128)HOSZP_QLIM) return false;
  rho = (long long)qq;
  return true;
}

// Scalar multiplication requantization: floor(2e * q * rho + 1/2), exact.
// 2e = M 2^E with M the 24-bit significand of the float 2e.
struct MulPlan {
  long long rho;
  long long M;
  int E;
};

__device__ __forceinline__ MulPlan mul_plan(float e, long long rho) {
  MulPlan p;
  p.rho = rho;
  const uint32_t bits = __float_as_uint(2.0f * e);  // normal: e >= FLT_MIN
  p.M = (long long)((bits & 0x7fffffu) | 0x800000u);
  p.E = (int)((bits >> 23) & 0xffu) - 127 - 23;
  return p;
}

// Returns q' and sets ovf when |q'| > HOSZP_QLIM.
__device__ __forceinline__ int mul_requant(int q, const MulPlan& p, bool& ovf) {
  const __int128 km = (__int128)((long long)q * p.rho) * p.M;  // |km| < 2^85
  __int128 r;
  if (p.E >= 0) {
    if (km == 0) return 0;
    if (p.E > 40) {
      ovf = true;
      return 0;
    }
    r = km << p.E;
  } else {
    const int sh = -p.E;
    if (sh >= 120) return 0;  // |2e q rho| < 2^-35
    const __int128 half = (__int128)1 << (sh - 1);
    r = (km + half) >> sh;  // arithmetic shift = floor
  }
  if (r > HOSZP_QLIM || r < -(__int128)HOSZP_QLIM) {
    ovf = true;
    return 0;
  }
  return (int)r;
}

// ---------------------------------------------------------------- workflow 1
// Stream copy (out of place) with every outlier transformed (negated or
// shifted by rho) and, for negation, every sign word inverted.
template <bool NEG>
__global__ void __launch_bounds__(512) k_meta(const uint8_t* c, uint64_t c_bytes, double s,
                                              uint8_t* out, uint64_t cap, uint64_t* out_bytes,
                                              Ws ws) {
  const Info h = parse_header(c, c_bytes);
  __shared__ int s_ok;
  __shared__ long long s_rho;
  if (threadIdx.x == 0) {
    int ok = h.ok;
    long long rho = 0;
    if (!h.ok) {
      if (blockIdx.x == 0) set_status(ws.status, HOSZP_ERR_FORMAT);
    } else if (h.size > cap) {
      ok = 0;
      if (blockIdx.x == 0) set_status(ws.status, HOSZP_ERR_CAPACITY);
    } else if (!NEG) {
      if (!quantize_scalar(s, h.eps_q, rho)) {
        ok = 0;
        if (blockIdx.x == 0) set_status(ws.status, HOSZP_ERR_RANGE);
      } else if ((long long)h.qbound + (rho < 0 ? -rho : rho) > HOSZP_QLIM) {
        ok = 0;
        if (blockIdx.x == 0) set_status(ws.status, HOSZP_ERR_OVERFLOW);
      }
    }
    s_ok = ok;
    s_rho = rho;
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  const long long rho = s_rho;
  if (ok) {
    const bool inplace = (out == c);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // outliers: 4 per thread step (section is 16-byte aligned)
    const int* src_o = reinterpret_cast<const int*>(c + h.o_out);
    int* dst_o = reinterpret_cast<int*>(out + h.o_out);
    for (uint64_t i = tid0; i < h.nb; i += stride) {
      const int o = src_o[i];
      dst_o[i] = NEG ? -o : (int)(o + rho);
    }
    if (NEG) {
      const uint64_t* src_s = reinterpret_cast<const uint64_t*>(c + h.o_sign);
      uint64_t* dst_s = reinterpret_cast<uint64_t*>(out + h.o_sign);
      for (uint64_t i = tid0; i < h.nnc; i += stride) dst_s[i] = ~src_s[i];
    }
    if (!inplace) {
      // rates (+ padding) and, for scalar addition, the sign words; then the planes
      const uint64_t* src = reinterpret_cast<const uint64_t*>(c);
      uint64_t* dst = reinterpret_cast<uint64_t*>(out);
      const uint64_t r0 = HOSZP_HEADER_BYTES / 8, r1 = h.o_out / 8;
      for (uint64_t i = r0 + tid0; i < r1; i += stride) dst[i] = src[i];
      const uint64_t pad0 = (h.o_out + 4 * h.nb + 7) / 8, pad1 = h.o_sign / 8;
      if ((h.nb & 1) && tid0 == 0) dst_o[h.nb] = src_o[h.nb];  // padding word half
      for (uint64_t i = pad0 + tid0; i < pad1; i += stride) dst[i] = src[i];
      const uint64_t w0 = (NEG ? h.o_plane : h.o_sign) / 8, w1 = h.size / 8;
      for (uint64_t i = w0 + tid0; i < w1; i += stride) dst[i] = src[i];
    }
  }
  // the header is written by the CTA that finishes last: in place, every other
  // CTA has parsed the input header by then
  if (launch_end_is_last(ws) && threadIdx.x == 0) {
    if (ok) {
      hoszp_header H = *reinterpret_cast<const hoszp_header*>(c);
      if (!NEG) H.qbound = (uint32_t)((long long)H.qbound + (rho < 0 ? -rho : rho));
      *reinterpret_cast<hoszp_header*>(out) = H;
      *out_bytes = h.size;
    } else {
      *out_bytes = 0;
    }
    launch_reset(ws);
  }
}

cudaError_t launch_negate(const Launch& lc, const uint8_t* c, uint64_t c_bytes, uint8_t* out,
                          uint64_t cap, uint64_t* out_bytes, Ws ws) {
  k_meta<true><<<persistent_grid(k_meta<true>, 512, lc.grid), 512, 0, lc.stream>>>(c, c_bytes, 0.0, out, cap, out_bytes, ws);
  return cudaGetLastError();
}

cudaError_t launch_add_scalar(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double s,
                              uint8_t* out, uint64_t cap, uint64_t* out_bytes, Ws ws) {
  k_meta<false><<<persistent_grid(k_meta<false>, 512, lc.grid), 512, 0, lc.stream>>>(c, c_bytes, s, out, cap, out_bytes, ws);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- shared re-encode step
// Octet of new deltas (|d| < 2^31) -> rate, sign byte, planes; the tile scan
// and the look-back on the output chain place them. Whole CTA.
struct OutTile {
  uint8_t rate[TILE];
  TileScan ts;
  unsigned long long pre[2];
};

__device__ __forceinline__ void encode_tile(uint64_t tile, uint64_t ntiles, uint64_t nb,
                                            const int d[8], int outlier, int g, int j,
                                            uint8_t* __restrict__ out, uint64_t cap, OutTile* s,
                                            Desc* chain, unsigned long long epoch, const Ws& ws,
                                            int& bad) {
  const uint64_t b = tile * TILE + g;
  uint32_t mag[8];
  uint32_t sb = 0;
#pragma unroll
  for (int t = 0; t < 8; t++) {
    mag[t] = (uint32_t)abs(d[t]);
    sb |= (d[t] < 0 ? 1u : 0u) << t;
  }
  const int rate = octet_rate(mag);
  if (j == 0) s->rate[g] = (b < nb) ? (uint8_t)rate : 0;
  __syncthreads();
  tile_scan(s->rate, &s->ts);
  tile_prefix(chain, (int64_t)tile, epoch, ws.status, s->ts.agg_nc, s->ts.agg_r, 0, s->pre);
  __syncthreads();
  const uint64_t NC = s->pre[0], RR = s->pre[1];
  const int r = (b < nb) ? rate : 0;
  if (b < nb && j == 0) {
    out[HOSZP_HEADER_BYTES + b] = (uint8_t)rate;
    reinterpret_cast<int*>(out + off_outlier(nb))[b] = outlier;
  }
  const uint64_t si = NC + s->ts.nc_excl[g];
  const uint64_t pi = RR + s->ts.r_excl[g];
  if (r > 0) {
    const uint64_t pos = off_sign(nb) + 8 * si + j;
    if (pos < cap) out[pos] = (uint8_t)sb;
    else bad = HOSZP_ERR_CAPACITY;
  }
  const int kmax = __reduce_max_sync(0xffffffffu, (r + 7) >> 3);
  const uint64_t lim = (pi < ws.staging_words) ? ws.staging_words - pi : 0;
  if (kmax > 0) encode_planes(mag, r, kmax, j, ws.staging + pi, lim);
  if (r > 0 && pi + r > ws.staging_words) bad = HOSZP_ERR_CAPACITY;
  if (tile == ntiles - 1 && threadIdx.x == 0) {
    ws.totals[0] = NC + s->ts.agg_nc;
    ws.totals[1] = RR + s->ts.agg_r;
  }
}

__device__ __forceinline__ void write_template(const Info& h, uint32_t qbound_fixed,
                                               const Ws& ws) {
  hoszp_header* H = ws.hdr;
  H->magic = HOSZP_MAGIC;
  H->version = HOSZP_VERSION;
  H->dtype = 0;
  H->ndims = (uint8_t)h.ndims;
  H->dims[0] = h.dims[0];
  H->dims[1] = h.dims[1];
  H->dims[2] = h.dims[2];
  H->eps_q = h.eps_q;
  H->n = h.n;
  H->eps = h.eps;
  H->nnc = 0;
  H->R = 0;
  H->qbound = qbound_fixed;
  H->block = HOSZP_BLOCK;
}

__device__ __forceinline__ void reduce_qmax(uint32_t qmax, const Ws& ws) {
  __shared__ uint32_t s_q[CTA / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qmax = max(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
  if ((threadIdx.x & 31) == 0) s_q[threadIdx.x >> 5] = qmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < CTA / 32; w++) qmax = max(qmax, s_q[w]);
    atomicMax(&ws.totals[2], (unsigned long long)qmax);
  }
}

// ---------------------------------------------------------------- scalar multiplication
__global__ void __launch_bounds__(CTA) k_mul_scalar(const uint8_t* __restrict__ c, uint64_t c_bytes,
                                                    double s, uint8_t* __restrict__ out,
                                                    uint64_t cap, Ws ws) {
  __shared__ InTile sin_;
  __shared__ OutTile sout;
  __shared__ unsigned int s_tile;
  __shared__ unsigned long long s_epoch;
  __shared__ long long s_rho;
  __shared__ int s_ok;
  const int tid = threadIdx.x, g = tid >> 3, j = tid & 7;
  const Info h = parse_header(c, c_bytes);
  int bad = 0;
  if (tid == 0) {
    s_epoch = launch_epoch(ws);
    int ok = h.ok;
    long long rho = 0;
    if (!h.ok) bad = HOSZP_ERR_FORMAT;
    else if (!quantize_scalar(s, h.eps_q, rho)) {
      ok = 0;
      bad = HOSZP_ERR_RANGE;
    } else if (cap < off_sign(h.nb)) {
      ok = 0;
      bad = HOSZP_ERR_CAPACITY;
    }
    s_ok = ok;
    s_rho = rho;
    if (blockIdx.x == 0) write_template(h, 0, ws);
  }
  __syncthreads();
  const unsigned long long epoch = s_epoch;
  const uint64_t ntiles = s_ok ? ntiles_of(h.nb) : 0;
  const MulPlan mp = mul_plan(h.ok ? h.eps_q : 1.0f, s_rho);
  uint32_t qmax = 0;
  bool ovf = false;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&ws.sync->ticket, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) break;
    in_tile_begin(c, h, tile, &sin_, ws.desc[0], epoch, ws.status, 0, bad);
    __syncthreads();
    if (tile == ntiles - 1 && tid == 0 &&
        (sin_.pre[0] + sin_.ts.agg_nc != h.nnc || sin_.pre[1] + sin_.ts.agg_r != h.R))
      bad = HOSZP_ERR_FORMAT;
    const BlockRef br = block_ref(c, h, tile, &sin_, g, j, bad);
    const int kmax = __reduce_max_sync(0xffffffffu, (br.rate + 7) >> 3);
    int d[8], q[8];
    octet_deltas(br, kmax, j, d);
    octet_values(br, d, j, q);
#pragma unroll
    for (int t = 0; t < 8; t++) {
      q[t] = (8 * j + t < br.len) ? mul_requant(q[t], mp, ovf) : 0;
      qmax = max(qmax, (uint32_t)abs(q[t]));
    }
    // Lorenzo on the new integers
    const int prev = __shfl_up_sync(0xffffffffu, q[7], 1, 8);
    const int outlier = __shfl_sync(0xffffffffu, q[0], tid & ~7);
    int nd[8];
#pragma unroll
    for (int t = 0; t < 8; t++) {
      int v = (t == 0) ? ((j == 0) ? 0 : q[0] - prev) : q[t] - q[t - 1];
      nd[t] = (8 * j + t < br.len) ? v : 0;
    }
    encode_tile(tile, ntiles, h.nb, nd, outlier, g, j, out, cap, &sout, ws.desc[1], epoch, ws,
                bad);
    __syncthreads();
  }
  if (ovf) bad = HOSZP_ERR_OVERFLOW;
  reduce_qmax(qmax, ws);
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && tid == 0) launch_reset(ws);
}

cudaError_t launch_mul_scalar(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double s,
                              uint8_t* out, uint64_t cap, Ws ws) {
  k_mul_scalar<<<persistent_grid(k_mul_scalar, CTA, lc.grid), CTA, 0, lc.stream>>>(c, c_bytes, s, out, cap, ws);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- element-wise addition
__global__ void __launch_bounds__(CTA) k_add(const uint8_t* __restrict__ a, uint64_t a_bytes,
                                             const uint8_t* __restrict__ b, uint64_t b_bytes,
                                             uint8_t* __restrict__ out, uint64_t cap, Ws ws) {
  __shared__ InTile sa, sb;
  __shared__ OutTile sout;
  __shared__ unsigned int s_tile;
  __shared__ unsigned long long s_epoch;
  __shared__ int s_ok;
  const int tid = threadIdx.x, g = tid >> 3, j = tid & 7;
  const Info ha = parse_header(a, a_bytes);
  const Info hb = parse_header(b, b_bytes);
  int bad = 0;
  if (tid == 0) {
    s_epoch = launch_epoch(ws);
    int ok = 0;
    if (!ha.ok || !hb.ok) bad = HOSZP_ERR_FORMAT;
    else if (ha.n != hb.n || __float_as_uint(ha.eps_q) != __float_as_uint(hb.eps_q))
      bad = HOSZP_ERR_MISMATCH;
    else if ((long long)ha.qbound + (long long)hb.qbound > HOSZP_QLIM)
      bad = HOSZP_ERR_OVERFLOW;
    else if (cap < off_sign(ha.nb))
      bad = HOSZP_ERR_CAPACITY;
    else
      ok = 1;
    s_ok = ok;
    if (blockIdx.x == 0) {
      write_template(ha, ok ? ha.qbound + hb.qbound : 0, ws);
      if (ok) atomicMax(&ws.totals[2], (unsigned long long)(ha.qbound + hb.qbound));
    }
  }
  __syncthreads();
  const unsigned long long epoch = s_epoch;
  const uint64_t ntiles = s_ok ? ntiles_of(ha.nb) : 0;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&ws.sync->ticket, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) break;
    // input chains: A with warp 0, B with warp 1
    {
      if (tid < TILE) {
        const uint64_t bb = tile * TILE + tid;
        uint8_t ra = (bb < ha.nb) ? a[HOSZP_HEADER_BYTES + bb] : 0;
        uint8_t rb = (bb < hb.nb) ? b[HOSZP_HEADER_BYTES + bb] : 0;
        if (ra > MAX_RATE || rb > MAX_RATE) {
          bad = HOSZP_ERR_FORMAT;
          ra = ra > MAX_RATE ? 0 : ra;
          rb = rb > MAX_RATE ? 0 : rb;
        }
        sa.rate[tid] = ra;
        sb.rate[tid] = rb;
      }
      __syncthreads();
      tile_scan(sa.rate, &sa.ts);
      tile_scan(sb.rate, &sb.ts);
      tile_prefix(ws.desc[0], (int64_t)tile, epoch, ws.status, sa.ts.agg_nc, sa.ts.agg_r, 0,
                  sa.pre);
      tile_prefix(ws.desc[1], (int64_t)tile, epoch, ws.status, sb.ts.agg_nc, sb.ts.agg_r, 1,
                  sb.pre);
      __syncthreads();
    }
    if (tile == ntiles - 1 && tid == 0 &&
        (sa.pre[0] + sa.ts.agg_nc != ha.nnc || sa.pre[1] + sa.ts.agg_r != ha.R ||
         sb.pre[0] + sb.ts.agg_nc != hb.nnc || sb.pre[1] + sb.ts.agg_r != hb.R))
      bad = HOSZP_ERR_FORMAT;
    const BlockRef ba = block_ref(a, ha, tile, &sa, g, j, bad);
    const BlockRef bbr = block_ref(b, hb, tile, &sb, g, j, bad);
    const int ka = __reduce_max_sync(0xffffffffu, (ba.rate + 7) >> 3);
    const int kb = __reduce_max_sync(0xffffffffu, (bbr.rate + 7) >> 3);
    int da[8], db[8], nd[8];
    octet_deltas(ba, ka, j, da);
    octet_deltas(bbr, kb, j, db);
#pragma unroll
    for (int t = 0; t < 8; t++) nd[t] = da[t] + db[t];
    encode_tile(tile, ntiles, ha.nb, nd, ba.outlier + bbr.outlier, g, j, out, cap, &sout,
                ws.desc[2], epoch, ws, bad);
    __syncthreads();
  }
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && tid == 0) launch_reset(ws);
}

cudaError_t launch_add(const Launch& lc, const uint8_t* a, uint64_t a_bytes, const uint8_t* b,
                       uint64_t b_bytes, uint8_t* out, uint64_t cap, Ws ws) {
  k_add<<<persistent_grid(k_add, CTA, lc.grid), CTA, 0, lc.stream>>>(a, a_bytes, b, b_bytes, out, cap, ws);
  return cudaGetLastError();
}

}  // namespace hz
