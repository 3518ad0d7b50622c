// Host runtime behind include/cachedconv.h: graph validation, the
// post-training causal reconfiguration analysis (section 3: right pad moved
// left; Eq. 2 stride alignment; cumulated lag; Eq. 3 branch alignment), the
// per-stream ring-buffer arena (cached padding, section 2.2), weight packing
// and the launch chain of one buffer.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/cachedconv.h"
#include "cc_internal.h"
#include "cc_runtime.h"

namespace cc {

thread_local std::string g_last_error;

cc_status fail(cc_status code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CC_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(CC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));           \
  } while (0)

static int64_t gcd64(int64_t a, int64_t b) { return b == 0 ? (a < 0 ? -a : a) : gcd64(b, a % b); }

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// Planning
// ---------------------------------------------------------------------------
static cc_status validate_and_analyze(Model& m) {
  const int n = (int)m.nodes.size();
  if (n < 2) return fail(CC_ERR_BAD_GRAPH, "a model needs an input node and at least one layer");
  for (int i = 0; i < n; ++i) {
    NodePlan& p = m.nodes[i];
    const cc_node_desc& d = p.d;
    if ((d.op == CC_OP_INPUT) != (i == 0))
      return fail(CC_ERR_BAD_GRAPH, "node %d: exactly node 0 must be the input", i);
    const int want = d.op == CC_OP_INPUT ? 0 : d.op == CC_OP_ADD ? 2 : d.op == CC_OP_HEADS ? 3 : 1;
    if (d.op < CC_OP_INPUT || d.op > CC_OP_HEADS)
      return fail(CC_ERR_BAD_GRAPH, "node %d: unknown op %d", i, d.op);
    if (d.n_inputs != want)
      return fail(CC_ERR_BAD_GRAPH, "node %d: op %d takes %d inputs, got %d", i, d.op, want, d.n_inputs);
    for (int q = 0; q < want; ++q)
      if (d.inputs[q] < 0 || d.inputs[q] >= i)
        return fail(CC_ERR_BAD_GRAPH, "node %d: input %d must be an earlier node", i, d.inputs[q]);
    if (d.act_in != CC_ACT_NONE && d.act_in != CC_ACT_LEAKY)
      return fail(CC_ERR_BAD_GRAPH, "node %d: unknown activation %d", i, d.act_in);
    if (d.c_out <= 0 || d.c_in <= 0) return fail(CC_ERR_BAD_GRAPH, "node %d: channels must be > 0", i);
    if (d.op == CC_OP_INPUT) {
      if (d.c_in != d.c_out) return fail(CC_ERR_BAD_GRAPH, "input node: c_in != c_out");
      p.rnum = 1;
      p.rden = 1;
      p.D = 0;
      continue;
    }
    const NodePlan& src = m.nodes[d.inputs[0]];
    for (int q = 0; q < want; ++q) {
      const NodePlan& s = m.nodes[d.inputs[q]];
      if (s.d.c_out != d.c_in)
        return fail(CC_ERR_BAD_GRAPH, "node %d: c_in %d != producer %d's c_out %d", i, d.c_in,
                    d.inputs[q], s.d.c_out);
      if (s.rnum * src.rden != src.rnum * s.rden)
        return fail(CC_ERR_BAD_GRAPH, "node %d: merged branches run at different rates", i);
    }
    if (d.op == CC_OP_CONV) {
      if (d.kernel < 1 || d.stride < 1 || d.dilation < 1 || d.pad_left < 0 || d.pad_right < 0)
        return fail(CC_ERR_BAD_GRAPH, "node %d: bad conv geometry", i);
      const int S = d.stride, R = d.pad_right;
      const int64_t Dc = src.D;
      // Eq. 2, read as the minimal extra delay in [0, S)
      p.Da = (int32_t)((S - (R + Dc) % S) % S);
      const int64_t total = Dc + R + p.Da;
      p.D = total / S;
      p.hist_need = d.pad_left + d.pad_right + p.Da;
      // streamable: the last output of a buffer may not need future input
      if ((int64_t)(d.kernel - 1) * d.dilation > p.hist_need + S - 1)
        return fail(CC_ERR_BAD_GRAPH,
                    "node %d: kernel span %d exceeds its left padding %d + stride - 1 "
                    "(the layer looks ahead; it cannot stream)",
                    i, (d.kernel - 1) * d.dilation, p.hist_need);
      const int64_t g = gcd64(src.rnum, src.rden * S);
      p.rnum = src.rnum / g;
      p.rden = src.rden * S / g;
    } else if (d.op == CC_OP_CONVT) {
      if (d.kernel < 1 || d.stride < 1 || d.kernel % d.stride != 0)
        return fail(CC_ERR_BAD_GRAPH, "node %d: convt kernel must be a multiple of its stride", i);
      if (d.crop < 0 || d.crop > d.kernel - d.stride)
        return fail(CC_ERR_BAD_GRAPH, "node %d: convt crop must lie in [0, K - S]", i);
      p.D = src.D * d.stride + d.crop;
      p.hist_need = d.kernel / d.stride - 1;
      const int64_t g = gcd64(src.rnum * d.stride, src.rden);
      p.rnum = src.rnum * d.stride / g;
      p.rden = src.rden / g;
    } else {
      if (d.c_in != d.c_out) return fail(CC_ERR_BAD_GRAPH, "node %d: merge keeps channels", i);
      if (d.act_in != CC_ACT_NONE) return fail(CC_ERR_BAD_GRAPH, "node %d: merges take no activation", i);
      int64_t dmax = 0;
      for (int q = 0; q < want; ++q) dmax = std::max(dmax, m.nodes[d.inputs[q]].D);
      for (int q = 0; q < want; ++q) p.A[q] = (int32_t)(dmax - m.nodes[d.inputs[q]].D);  // Eq. 3
      p.D = dmax;
      p.rnum = src.rnum;
      p.rden = src.rden;
    }
  }
  // steps: lcm of rate denominators
  int64_t ips = 1;
  for (auto& p : m.nodes) ips = ips / gcd64(ips, p.rden) * p.rden;
  if (ips > (1 << 24)) return fail(CC_ERR_BAD_GRAPH, "model step of %lld input frames is too long", (long long)ips);
  m.in_per_step = (int32_t)ips;
  for (auto& p : m.nodes) p.u = (int32_t)(ips * p.rnum / p.rden);
  // engines: contractions whose input channels fill whole 64-wide K slices
  // run on tensor cores in the low-precision modes
  for (auto& p : m.nodes)
    p.engine = (m.dtype != CC_F32 && (p.d.op == CC_OP_CONV || p.d.op == CC_OP_CONVT) &&
                p.d.c_in % 64 == 0 && p.d.c_out % 8 == 0)
                   ? 1
                   : 0;
  // history each producer keeps = max over its consumers' needs, per view
  for (int i = 0; i < n; ++i) {
    const NodePlan& c = m.nodes[i];
    const cc_node_desc& d = c.d;
    for (int q = 0; q < d.n_inputs; ++q) {
      NodePlan& src = m.nodes[d.inputs[q]];
      src.consumers.push_back(i);
      const bool merge = d.op == CC_OP_ADD || d.op == CC_OP_HEADS;
      const int need = merge ? c.A[q] : c.hist_need;
      const int v = (!merge && c.engine == 1) ? 1 + d.act_in : 0;
      src.keep = std::max(src.keep, need);
      src.keep_view[v] = std::max(src.keep_view[v], need);
      src.used_view[v] = true;
    }
  }
  return CC_OK;
}

// Residual adds are folded into the epilogue of the layer that finishes their
// last branch when that layer has no other consumer and is not delayed.
static void plan_fusion(Model& m) {
  const int n = (int)m.nodes.size();
  for (int i = 0; i < n; ++i) {
    NodePlan& add = m.nodes[i];
    if (add.d.op != CC_OP_ADD) continue;
    for (int k = 1; k >= 0; --k) {
      const int pk = add.d.inputs[k], other = add.d.inputs[1 - k];
      NodePlan& prod = m.nodes[pk];
      if ((prod.d.op == CC_OP_CONV || prod.d.op == CC_OP_CONVT) && prod.consumers.size() == 1 &&
          add.A[k] == 0 && other < pk && prod.fused_add < 0) {
        prod.fused_add = i;
        prod.fused_skip = other;
        prod.fused_skip_A = add.A[1 - k];
        add.fused = true;
        break;
      }
    }
  }
}

// Sibling tensor-core convolutions (stride 1, dilation 1) that read the same
// input view and whose outputs are read in FP32 only run as one contraction:
// M = the members' channels side by side (at most 128), the windows
// right-aligned (a member with less history starts its taps later; the taps
// in front of them are zero), one FP32 ring whose rows hold every member's
// channels (each member's view points at its channels).
static void plan_siblings(Model& m) {
  if (!m.merge_siblings) return;
  const int n = (int)m.nodes.size();
  auto eligible = [&](const NodePlan& p) {
    return p.d.op == CC_OP_CONV && p.engine == 1 && p.d.stride == 1 && p.d.dilation == 1 && p.fused_add < 0 &&
           p.group_leader < 0 && !p.consumers.empty() && !p.used_view[1] && !p.used_view[2] &&
           p.d.c_out % 8 == 0;
  };
  for (int i = 0; i < n; ++i) {
    NodePlan& lead = m.nodes[i];
    if (!eligible(lead)) continue;
    std::vector<int> g{i};
    int32_t ctot = lead.d.c_out;
    for (int j = i + 1; j < n; ++j) {
      const NodePlan& q = m.nodes[j];
      if (!eligible(q) || q.d.inputs[0] != lead.d.inputs[0] || q.d.act_in != lead.d.act_in ||
          q.d.c_in != lead.d.c_in || ctot + q.d.c_out > 128)
        continue;
      g.push_back(j);
      ctot += q.d.c_out;
    }
    if (g.size() < 2) continue;
    int32_t hist = 0, taps = 0;
    for (int k : g) hist = std::max(hist, m.nodes[k].hist_need);
    for (int k : g) taps = std::max(taps, hist - m.nodes[k].hist_need + m.nodes[k].d.kernel);
    int32_t off = 0;
    for (int k : g) {
      m.nodes[k].group_leader = i;
      m.nodes[k].choff = off;
      off += m.nodes[k].d.c_out;
    }
    lead.group = g;
    lead.group_taps = taps;
    lead.group_hist = hist;
  }
}

// Residual units on tensor cores: a stride-1 conv whose only consumer is a
// 1x1 conv with a fused residual (and no history) run as one launch; the
// intermediate never leaves the chip.  Units of up to 128 channels fit one
// 128-row tile; units of up to 256 channels run as clusters of two M tiles
// that exchange their halves of the intermediate in distributed shared
// memory (one CTA per SM, so only in models of at most 256 streams, whose
// launches fit one wave).  A model built without unit fusion runs the same
// layers unsplit, so that both forms sum in the same order.
static void plan_units(Model& m) {
  const int n = (int)m.nodes.size();
  for (int i = 0; i < n; ++i) {
    NodePlan& p = m.nodes[i];
    if (p.d.op != CC_OP_CONV || p.engine != 1 || p.d.stride != 1 || p.fused_add >= 0 ||
        p.consumers.size() != 1 || p.group_leader >= 0)
      continue;
    const int qi = p.consumers[0];
    NodePlan& q = m.nodes[qi];
    if (q.d.op != CC_OP_CONV || q.engine != 1 || q.d.kernel != 1 || q.d.stride != 1 || q.hist_need != 0 ||
        q.fused_add < 0 || q.unit_fused)
      continue;
    if (q.d.c_in != p.d.c_out || q.d.c_out != p.d.c_out) continue;
    const bool wide = p.M > 128 || q.M > 128 || q.Kt > 128;
    if (p.M > 256 || q.M > 256 || q.Kt > 256) continue;
    if (wide && m.max_streams > 256) continue;
    if (!m.fuse_units) {
      if (wide) p.no_split = q.no_split = true;
      continue;
    }
    p.unit_next = qi;
    q.unit_fused = true;
  }
}

// Split-K for tensor-core layers whose tiles at full capacity (max_streams,
// one step) fill few SMs and whose K is long: clusters of 4 or 2 CTAs share a
// tile.  Chosen from the layer and the capacity only, so that every batch
// runs the same arithmetic; fused residual units run unsplit.
static void plan_ksplit(Model& m) {
  for (auto& p : m.nodes) {
    p.ksplit = 1;
    if (p.engine != 1 || p.unit_next >= 0 || p.unit_fused || p.no_split) continue;
    if (p.group_leader >= 0 && p.group_leader != (int)(&p - m.nodes.data())) continue;
    const int nk = p.Kt / 64, mt = p.Mpad / 128;
    const int64_t cols =
        (int64_t)m.max_streams * (p.d.op == CC_OP_CONVT ? m.nodes[p.d.inputs[0]].u : p.u);
    const int64_t ctas = (cols + 127) / 128 * mt;
    p.ksplit = (ctas * 4 <= 148 && nk >= 8) ? 4 : (ctas * 2 <= 148 && nk >= 4) ? 2 : 1;
  }
}

// The cached state as ring regions: every view's kept rows (one region per
// ring: a sibling group's shared FP32 ring keeps its members' largest history).
static cc_status plan_state(Model& m) {
  m.state_regions.clear();
  std::map<int64_t, size_t> by_off;
  for (const NodePlan& p : m.nodes) {
    if (!p.has_ring) continue;
    for (int v = 0; v < 3; ++v) {
      const Ring& r = p.view[v];
      if (!r.rows || !p.keep_view[v]) continue;
      const int32_t elem = v == 0 ? 4 : 2;
      auto it = by_off.find(r.off);
      if (it != by_off.end()) {
        m.state_regions[it->second].keep = std::max(m.state_regions[it->second].keep, p.keep_view[v]);
        continue;
      }
      Model::StateRegion g{};
      g.off = r.off;
      g.rows = r.rows;
      g.pre = r.pre;
      g.row_bytes = r.chans * elem;
      g.keep = p.keep_view[v];
      g.u = r.u;
      if (g.row_bytes % 4) return fail(CC_ERR_STATE, "state row of %d bytes is not a multiple of 4", g.row_bytes);
      by_off[r.off] = m.state_regions.size();
      m.state_regions.push_back(g);
    }
  }
  m.snapshot_bytes = 16;
  for (const auto& g : m.state_regions) m.snapshot_bytes += (size_t)g.keep * g.row_bytes;
  m.snapshot_bytes = align_up(m.snapshot_bytes, 16);  // every stream's record 16-byte aligned in a batch buffer
  return CC_OK;
}

static size_t lcm_size(size_t a, size_t b) {
  size_t x = a, y = b;
  while (y) {
    const size_t t = x % y;
    x = y;
    y = t;
  }
  return a / x * b;
}

// Low-precision views are aligned to their row pitch (and the slot size to
// every such pitch) so that a single 2D tensor map over the arena addresses
// the rows of that view in every stream's slot.  Their rings hold whole
// steps (R a multiple of u, so a one-step call never crosses the ring's end)
// and at least four times the kept history, whose mirror sits before row 0:
// the mirrored tail costs at most a quarter of the view's stores.
static cc_status plan_arena(Model& m) {
  size_t off = 0, state = 0, slot_align = 256;
  const int n = (int)m.nodes.size();
  for (int i = 0; i < n; ++i) {
    NodePlan& p = m.nodes[i];
    const bool needs_ring = !p.consumers.empty() && p.fused_add < 0;
    if (!needs_ring) continue;
    p.has_ring = true;
    if (p.group_leader >= 0) {
      // one FP32 ring for the sibling group, made when the leader comes by
      NodePlan& lead = m.nodes[p.group_leader];
      if (p.group_leader == i) {
        int64_t rows = 0;
        int32_t chans = 0;
        for (int k : lead.group) {
          const NodePlan& q = m.nodes[k];
          rows = std::max(rows, (int64_t)q.keep_view[0] + (int64_t)q.u * m.max_steps);
          chans += q.d.c_out;
        }
        if (rows >= (1ll << 30)) return fail(CC_ERR_NO_MEMORY, "ring of node %d too long", i);
        Ring r{};
        r.rows = (int32_t)rows;
        r.chans = chans;
        r.u = p.u;
        r.dtype = kDtF32;
        r.off = (int64_t)off;
        off = align_up(off + (size_t)rows * chans * 4, 256);
        lead.view[0] = r;
      }
      Ring r = lead.view[0];
      r.choff = p.choff;
      p.view[0] = r;
      state += (size_t)p.keep_view[0] * p.d.c_out * 4;
      continue;
    }
    for (int v = 0; v < 3; ++v) {
      if (!p.used_view[v]) continue;
      Ring& r = p.view[v];
      const int64_t keep = p.keep_view[v];
      int64_t rows = keep + (int64_t)p.u * m.max_steps;
      r.chans = p.d.c_out;
      r.u = p.u;
      r.dtype = v == 0 ? kDtF32 : m.lp_dtype;
      r.pre = 0;
      const size_t elem = v == 0 ? 4 : 2;
      if (v > 0) {
        const size_t pitch = (size_t)r.chans * elem;
        rows = std::max(rows, 4 * keep);
        rows = (rows + p.u - 1) / p.u * p.u;
        r.pre = (int32_t)keep;
        off = align_up(off, lcm_size(256, pitch));
        off += (size_t)r.pre * pitch;
        slot_align = lcm_size(slot_align, pitch);
      }
      if (rows >= (1ll << 30)) return fail(CC_ERR_NO_MEMORY, "ring of node %d too long", i);
      r.rows = (int32_t)rows;
      r.off = (int64_t)off;
      off = align_up(off + (size_t)r.rows * r.chans * elem, 256);
      state += (size_t)p.keep_view[v] * p.d.c_out * elem;
    }
  }
  m.slot_bytes = std::max<size_t>(align_up(off, slot_align), slot_align);
  m.state_bytes = state;
  return CC_OK;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Low-precision tensor-core copy of a packed FP32 GEMM operand: rows scaled
// to max |w| = 1 (the scale is re-applied in FP32 by the epilogue), padded to
// 128-row tiles, described by a TMA map of 128 x 64 boxes, 128-byte swizzle.
static cc_status upload_tc_operand(Model& m, NodePlan& p, const std::vector<float>& A) {
  p.Mpad = (p.M + 127) / 128 * 128;
  std::vector<uint16_t> lp((size_t)p.Mpad * p.Kt, 0);
  std::vector<float> scale(p.Mpad, 1.0f);
  for (int r = 0; r < p.M; ++r) {
    float mx = 0.f;
    for (int k = 0; k < p.Kt; ++k) mx = std::max(mx, std::fabs(A[(size_t)r * p.Kt + k]));
    const float sc = mx > 0.f ? mx : 1.0f;
    scale[r] = sc;
    for (int k = 0; k < p.Kt; ++k) {
      const float x = A[(size_t)r * p.Kt + k] / sc;
      uint16_t bits;
      if (m.lp_dtype == kDtBF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        std::memcpy(&bits, &h, 2);
      } else {
        const __half h = __float2half_rn(x);
        std::memcpy(&bits, &h, 2);
      }
      lp[(size_t)r * p.Kt + k] = bits;
    }
  }
  CC_CUDA(cudaMalloc(&p.dA_lp, lp.size() * 2));
  CC_CUDA(cudaMemcpy(p.dA_lp, lp.data(), lp.size() * 2, cudaMemcpyHostToDevice));
  // the same operand as contiguous 128 x 64 blocks (16 KB), block (mt, kc) at
  // (mt * Kt/64 + kc) * 16 KB; inside a block row r's 16-byte chunk c sits at
  // r*128 + ((c ^ (r & 7)) * 16): the shared-memory image of a 128-byte-swizzled
  // K-major tile, so one bulk copy reproduces it.  With M <= 64, rows 64..127
  // repeat rows 0..63 (TcArgs::mdup): the padding rows compute the same
  // results, which the epilogue warps of the upper lane quarters store
  {
    const int nk = p.Kt / 64, mt_n = p.Mpad / 128;
    std::vector<uint16_t> tiled(lp.size());
    for (int mt = 0; mt < mt_n; ++mt)
      for (int kc = 0; kc < nk; ++kc) {
        uint16_t* blk = tiled.data() + ((size_t)mt * nk + kc) * 128 * 64;
        for (int r = 0; r < 128; ++r) {
          const int rs = p.M <= 64 ? (r & 63) : r;
          for (int c = 0; c < 8; ++c)
            std::memcpy(blk + r * 64 + ((c ^ (r & 7)) * 8),
                        lp.data() + (size_t)(mt * 128 + rs) * p.Kt + kc * 64 + c * 8, 16);
        }
      }
    CC_CUDA(cudaMalloc(&p.dA_tiled, tiled.size() * 2));
    CC_CUDA(cudaMemcpy(p.dA_tiled, tiled.data(), tiled.size() * 2, cudaMemcpyHostToDevice));
  }
  CC_CUDA(cudaMalloc(&p.dscale, scale.size() * sizeof(float)));
  CC_CUDA(cudaMemcpy(p.dscale, scale.data(), scale.size() * sizeof(float), cudaMemcpyHostToDevice));
  m.weight_bytes += lp.size() * 2;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return fail(CC_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[2] = {(cuuint64_t)p.Kt, (cuuint64_t)p.Mpad};
  const cuuint64_t strides[1] = {(cuuint64_t)p.Kt * 2};
  const cuuint32_t box[2] = {64, 128};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(reinterpret_cast<CUtensorMap*>(p.tmap),
                         m.lp_dtype == kDtBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                         2, p.dA_lp, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CC_ERR_CUDA, "tensor map encoding failed (%d)", (int)r);
  return CC_OK;
}

// Tensor map of a tensor-core layer's input view: the whole arena as rows of
// C low-precision elements, one-row boxes of 64 elements, 128-byte swizzle.
static cc_status encode_gather_maps(Model& m) {
  EncodeTiledFn enc = encode_tiled();
  for (auto& p : m.nodes) {
    if (p.engine != 1) continue;
    const Ring& in = m.nodes[p.d.inputs[0]].view[1 + p.d.act_in];
    const size_t pitch = (size_t)in.chans * 2;
    if (!enc) return fail(CC_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (m.slot_bytes % pitch || in.off % pitch) return fail(CC_ERR_STATE, "arena view not row aligned");
    const uint64_t rows = (uint64_t)m.max_streams * (m.slot_bytes / pitch);
    if (rows >= (1ull << 31)) return fail(CC_ERR_NO_MEMORY, "arena too large for 32-bit row indices");
    p.in_rows_per_slot = (int32_t)(m.slot_bytes / pitch);
    p.in_row_off = (int32_t)(in.off / pitch);
    const cuuint64_t dims[2] = {(cuuint64_t)in.chans, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {64, 1};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(reinterpret_cast<CUtensorMap*>(p.tmapB),
                           m.lp_dtype == kDtBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                           2, m.arena, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CC_ERR_CUDA, "gather tensor map encoding failed (%d)", (int)r);
    // box maps: the view of every slot as [slot][pre + R rows][C]; box i covers
    // 2^i consecutive rows of 2^(7-i) consecutive slots (128 rows in all).  A
    // shape the driver rejects (a box larger than the view) stays unused.
    const cuuint64_t d3[3] = {(cuuint64_t)in.chans, (cuuint64_t)(in.pre + in.rows), (cuuint64_t)m.max_streams};
    const cuuint64_t s3[2] = {(cuuint64_t)pitch, (cuuint64_t)m.slot_bytes};
    const cuuint32_t e3[3] = {1, 1, 1};
    for (int li = 0; li < 8; ++li) {
      const cuuint32_t b3[3] = {64, 1u << li, 1u << (7 - li)};
      p.tmapT_ok[li] = false;
      if (b3[1] > d3[1] || b3[2] > d3[2]) continue;
      const CUresult r3 = enc(reinterpret_cast<CUtensorMap*>(p.tmapT[li]),
                              m.lp_dtype == kDtBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                              3, m.arena + in.off - (int64_t)in.pre * (int64_t)pitch, d3, s3, b3, e3,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      p.tmapT_ok[li] = r3 == CUDA_SUCCESS;
    }
  }
  return CC_OK;
}

static cc_status pack_and_upload(Model& m, const float* const* weights, const float* const* biases) {
  for (int i = 0; i < (int)m.nodes.size(); ++i) {
    NodePlan& p = m.nodes[i];
    const cc_node_desc& d = p.d;
    if (d.op != CC_OP_CONV && d.op != CC_OP_CONVT) continue;
    if (!weights || !weights[i]) return fail(CC_ERR_INVALID_ARG, "node %d: missing weights", i);
    if (d.has_bias && (!biases || !biases[i])) return fail(CC_ERR_INVALID_ARG, "node %d: missing bias", i);
    std::vector<float> A;
    const float* w = weights[i];
    if (p.group_leader >= 0) {
      if (p.group_leader != i) continue;  // computed by the leader
      // [sum c_out][taps * c_in]: member k's tap j at merged tap j + (hist - hist_k)
      int32_t M = 0;
      for (int k : p.group) M += m.nodes[k].d.c_out;
      p.taps = p.group_taps;
      p.phases = 1;
      p.M = M;
      p.Kt = p.group_taps * d.c_in;
      A.assign((size_t)p.M * p.Kt, 0.f);
      std::vector<float> bias(M, 0.f);
      bool any_bias = false;
      for (int k : p.group) {
        const NodePlan& q = m.nodes[k];
        if (!weights[k]) return fail(CC_ERR_INVALID_ARG, "node %d: missing weights", k);
        if (q.d.has_bias && (!biases || !biases[k])) return fail(CC_ERR_INVALID_ARG, "node %d: missing bias", k);
        const int shift = p.group_hist - q.hist_need;
        for (int o = 0; o < q.d.c_out; ++o) {
          for (int c = 0; c < d.c_in; ++c)
            for (int j = 0; j < q.d.kernel; ++j)
              A[(size_t)(q.choff + o) * p.Kt + (size_t)(j + shift) * d.c_in + c] =
                  weights[k][((size_t)o * d.c_in + c) * q.d.kernel + j];
          if (q.d.has_bias) {
            bias[q.choff + o] = biases[k][o];
            any_bias = true;
          }
        }
      }
      cc_status s = upload_tc_operand(m, p, A);
      if (s) return s;
      if (any_bias) {
        CC_CUDA(cudaMalloc(&p.dbias, M * sizeof(float)));
        CC_CUDA(cudaMemcpy(p.dbias, bias.data(), M * sizeof(float), cudaMemcpyHostToDevice));
      }
      continue;
    }
    if (d.op == CC_OP_CONV) {
      // trained [c_out][c_in][K] -> [c_out][K][c_in]: a K-slice is one tap
      p.taps = d.kernel;
      p.phases = 1;
      p.M = d.c_out;
      p.Kt = d.kernel * d.c_in;
      A.resize((size_t)p.M * p.Kt);
      for (int o = 0; o < d.c_out; ++o)
        for (int c = 0; c < d.c_in; ++c)
          for (int k = 0; k < d.kernel; ++k)
            A[(size_t)o * p.Kt + (size_t)k * d.c_in + c] = w[((size_t)o * d.c_in + c) * d.kernel + k];
    } else {
      // trained [c_in][c_out][K] -> polyphase rows (phase, n), columns (tap k', c):
      // y[qS + phase] = sum_j w[c][n][phase + jS] x[q - j], tap k' = T - 1 - j
      const int S = d.stride, T = d.kernel / S;
      p.taps = T;
      p.phases = S;
      p.M = S * d.c_out;
      p.Kt = T * d.c_in;
      A.resize((size_t)p.M * p.Kt);
      for (int ph = 0; ph < S; ++ph)
        for (int o = 0; o < d.c_out; ++o)
          for (int kp = 0; kp < T; ++kp)
            for (int c = 0; c < d.c_in; ++c) {
              const int k = ph + (T - 1 - kp) * S;
              A[(size_t)(ph * d.c_out + o) * p.Kt + (size_t)kp * d.c_in + c] =
                  w[((size_t)c * d.c_out + o) * d.kernel + k];
            }
    }
    if (p.engine == 1) {
      cc_status s = upload_tc_operand(m, p, A);
      if (s) return s;
    } else {
      CC_CUDA(cudaMalloc(&p.dA, A.size() * sizeof(float)));
      CC_CUDA(cudaMemcpy(p.dA, A.data(), A.size() * sizeof(float), cudaMemcpyHostToDevice));
      m.weight_bytes += A.size() * sizeof(float);
    }
    if (d.has_bias) {
      CC_CUDA(cudaMalloc(&p.dbias, d.c_out * sizeof(float)));
      CC_CUDA(cudaMemcpy(p.dbias, biases[i], d.c_out * sizeof(float), cudaMemcpyHostToDevice));
    }
  }
  return CC_OK;
}

// ---------------------------------------------------------------------------
// One launch chain: `steps` model steps for every stream of `batch`.
// ---------------------------------------------------------------------------
cc_status Model::run_chain(const Batch& batch, const float* in, int64_t in_stride, float* out,
                           int64_t out_stride, int32_t steps, cudaStream_t st) {
  const int n = (int)nodes.size();
  const int last = n - 1;
  auto begin = [&](int i) -> cc_status {
    if (timing_on) {
      TimingRec r;
      r.node = i;
      CC_CUDA(take_event(&r.start));
      CC_CUDA(take_event(&r.stop));
      CC_CUDA(cudaEventRecord(r.start, st));
      timing_recs.push_back(r);
    }
    return CC_OK;
  };
  auto end = [&]() -> cc_status {
    if (timing_on) CC_CUDA(cudaEventRecord(timing_recs.back().stop, st));
    return CC_OK;
  };
  auto views_of = [&](int wi) {
    OutViews o{};
    const NodePlan& w = nodes[wi];
    o.f32 = w.view[0];
    o.lp[0] = w.view[1];
    o.lp[1] = w.view[2];
    o.ext = wi == last ? out : nullptr;
    o.ext_stride = out_stride;
    return o;
  };
  // launch index at which each node's values were written (a fused add's by
  // its producer's launch): a residual written two or more launches before
  // its reader is final when the reader starts (see k_conv_tc)
  std::vector<int> made_at(n, -1);
  int launches = 0;
  bool advanced = false;  // the step counters were advanced by the last launch
  for (int i = 0; i < n; ++i) {
    NodePlan& p = nodes[i];
    const cc_node_desc& d = p.d;
    if (d.op == CC_OP_INPUT) {
      made_at[i] = launches++;
      InputArgs a{};
      a.src = in;
      a.src_stride = in_stride;
      a.manip = in_manip;
      a.ncols = p.u * steps;
      a.chans = d.c_out;
      a.out_u = p.u;
      a.out = views_of(i);
      a.batch = batch;
      cc_status s = begin(i);
      if (s) return s;
      CC_CUDA(launch_input(a, st));
      if ((s = end())) return s;
      continue;
    }
    if (d.op == CC_OP_ADD && p.fused) continue;
    if (p.unit_fused) continue;  // computed by its producer's fused launch
    if (p.group_leader >= 0 && p.group_leader != i) continue;  // computed by its group's leader
    // a fused residual unit writes the 1x1 conv's (and its fused add's) output
    const int qi = p.unit_next;
    const NodePlan* q = qi >= 0 ? &nodes[qi] : nullptr;
    const NodePlan& r = q ? *q : p;  // the conv whose output this launch stores
    // the node whose output this launch writes (a fused add writes for its conv)
    const int wi = (r.d.op == CC_OP_CONV || r.d.op == CC_OP_CONVT) && r.fused_add >= 0 ? r.fused_add : (q ? qi : i);
    const NodePlan& w = nodes[wi];
    if (wi != last && !w.has_ring) continue;  // dead branch
    const OutViews ov = views_of(wi);
    const int this_launch = launches++;
    made_at[i] = made_at[wi] = this_launch;
    if (q) made_at[qi] = this_launch;
    for (int k : p.group) made_at[k] = this_launch;
    cc_status s = begin(i);
    if (s) return s;
    if (d.op == CC_OP_CONV || d.op == CC_OP_CONVT) {
      const NodePlan& src = nodes[d.inputs[0]];
      const bool convt = d.op == CC_OP_CONVT;
      const int32_t ncols = convt ? src.u * steps : p.u * steps;
      const int32_t dil = convt ? 1 : d.dilation, stride = convt ? 1 : d.stride;
      if (p.engine == 1) {
        TcArgs a{};
        a.A_tiled = p.dA_tiled;
        a.scale = p.dscale;
        a.bias = p.dbias;
        a.M = p.M;
        a.Kt = p.Kt;
        a.taps = p.taps;
        a.cin = d.c_in;
        a.dil = dil;
        a.stride = stride;
        a.hist = p.group.empty() ? p.hist_need : p.group_hist;
        a.ncols = ncols;
        a.cout = p.group.empty() ? d.c_out : p.M;
        a.phases = p.phases;
        a.out_u = w.u;
        a.in = src.view[1 + d.act_in];
        a.in_rows_per_slot = p.in_rows_per_slot;
        a.in_row_off = p.in_row_off;
        a.out = ov;
        if (r.fused_add >= 0) {
          a.has_skip = 1;
          a.skip = nodes[r.fused_skip].view[0];
          a.skip_A = r.fused_skip_A;
          const int sm = made_at[r.fused_skip];
          a.skip_early = sm >= 0 && sm <= this_launch - 2;
        }
        if (q) {
          a.A2_tiled = q->dA_tiled;
          a.scale2 = q->dscale;
          a.bias2 = q->dbias;
          a.k2 = q->Kt / 64;
          a.act2 = q->d.act_in;
        }
        a.batch = batch;
        a.err = err;
        a.wait_ns = wait_ns;
        a.withhold = withhold;
        // 3D window boxes: stride 1 and a box of min(ncols, 128) frames that
        // tiles the 128-column halves of a tile exactly
        int li = -1;
        if (stride == 1 && (128 % ncols == 0 || ncols % 128 == 0)) {
          li = 0;
          while ((1 << li) < std::min(ncols, 128)) ++li;
          if (!p.tmapT_ok[li]) li = -1;
        }
        a.box_ok = li >= 0;
        a.ksplit = p.ksplit;
        a.deep_ok = max_streams <= 256;
        a.mdup = p.M <= 64 && (!q || q->M <= 64);  // the tiles repeat their rows (upload_tc_operand)
        const int bn = tile_n_for(p, (int64_t)batch.count * ncols);
        CC_CUDA(launch_conv_tc(li >= 0 ? p.tmapT[li] : p.tmapB, p.tmapB, a, bn, st));
      } else {
        ConvArgs a{};
        a.A = p.dA;
        a.bias = p.dbias;
        a.M = p.M;
        a.Kt = p.Kt;
        a.taps = p.taps;
        a.cin = d.c_in;
        a.act = d.act_in;
        a.cout = d.c_out;
        a.phases = p.phases;
        a.dil = dil;
        a.stride = stride;
        a.hist = p.hist_need;
        a.ncols = ncols;
        a.out_u = w.u;
        a.in = src.view[0];
        a.out = ov;
        if (p.fused_add >= 0) {
          a.has_skip = 1;
          a.skip = nodes[p.fused_skip].view[0];
          a.skip_A = p.fused_skip_A;
        }
        a.batch = batch;
        // the chain's last launch advances the step counters itself when it can
        if (wi == last && conv_f32_can_advance(a)) {
          a.advance = steps;
          advanced = true;
        }
        CC_CUDA(launch_conv_f32(a, st));
      }
    } else if (d.op == CC_OP_ADD) {
      AddArgs a{};
      for (int q = 0; q < 2; ++q) {
        a.in[q] = nodes[d.inputs[q]].view[0];
        a.A[q] = p.A[q];
      }
      a.ncols = p.u * steps;
      a.chans = d.c_out;
      a.out_u = p.u;
      a.out = ov;
      a.batch = batch;
      CC_CUDA(launch_add(a, st));
    } else {
      HeadsArgs a{};
      for (int q = 0; q < 3; ++q) {
        a.in[q] = nodes[d.inputs[q]].view[0];
        a.A[q] = p.A[q];
      }
      a.delay = p.D;
      a.bands = d.c_out;
      a.ncols = p.u * steps;
      a.noise = noise;
      a.out_u = p.u;
      a.out = ov;
      a.batch = batch;
      CC_CUDA(launch_heads(a, st));
    }
    if ((s = end())) return s;
  }
  if (!advanced) {
    CC_CUDA(launch_advance(batch, steps, st));
    ++launches;
  }
  last_chain_launches = launches;
  return CC_OK;
}

int32_t Model::tile_n_for(const NodePlan& p, int64_t n_cols) const {
  if (force_tile_n) return force_tile_n;
  auto it = p.tile_n.find(n_cols);
  if (it != p.tile_n.end()) return it->second;
  return tc_tile_n(n_cols, p.Mpad / 128);
}

// Project autotuner: times one launch chain with every tensor-core layer on
// 128-column tiles and one with 256-column tiles (CUDA events around each
// launch), and keeps the faster shape per layer for this launch width.  The
// chain runs on the given slots, whose rings and step counters it advances:
// callers pass scratch slots.
// Tile width per tensor-core layer for one launch width: each candidate (128
// and 256 columns) is warmed up, then timed per layer in kTuneRounds rounds
// that alternate the candidates (so a clock or occupancy drift does not favour
// one), and each layer keeps the candidate with the smaller per-round minimum.
cc_status Model::autotune(const int32_t* d_slots, int32_t count, const float* in, int64_t in_stride,
                          float* out, int64_t out_stride, cudaStream_t st) {
  constexpr int kTuneRounds = 3;
  const int n = (int)nodes.size();
  const int32_t cands[2] = {128, 256};
  std::vector<double> best_ms[2] = {std::vector<double>(n, 1e30), std::vector<double>(n, 1e30)};
  const Batch b = batch_for(d_slots, count);
  for (int c = 0; c < 2; ++c) {  // warm up (kernel attributes, caches)
    force_tile_n = cands[c];
    cc_status s = run_chain(b, in, in_stride, out, out_stride, 1, st);
    force_tile_n = 0;
    if (s) return s;
  }
  CC_CUDA(cudaStreamSynchronize(st));
  for (int round = 0; round < kTuneRounds; ++round)
    for (int c = 0; c < 2; ++c) {
      force_tile_n = cands[c];
      timing_on = true;
      timing_recs.clear();
      event_pool_used = 0;
      cc_status s = run_chain(b, in, in_stride, out, out_stride, 1, st);
      timing_on = false;
      force_tile_n = 0;
      if (s) return s;
      CC_CUDA(cudaStreamSynchronize(st));
      std::vector<double> ms(n, 0.0);
      for (auto& rec : timing_recs) {
        float t = 0.f;
        CC_CUDA(cudaEventElapsedTime(&t, rec.start, rec.stop));
        ms[rec.node] += t;
      }
      for (int i = 0; i < n; ++i) best_ms[c][i] = std::min(best_ms[c][i], ms[i]);
    }
  timing_recs.clear();
  event_pool_used = 0;
  for (int i = 0; i < n; ++i) {
    NodePlan& p = nodes[i];
    if (p.engine != 1) continue;
    const NodePlan& src = nodes[p.d.inputs[0]];
    const int64_t cols = (int64_t)count * (p.d.op == CC_OP_CONVT ? src.u : p.u);
    p.tile_n[cols] = best_ms[1][i] < best_ms[0][i] ? cands[1] : cands[0];
  }
  drop_chain_graphs();  // they were captured with the previous tile shapes
  return CC_OK;
}

cudaError_t Model::take_event(cudaEvent_t* ev) {
  if (event_pool_used < event_pool.size()) {
    *ev = event_pool[event_pool_used++];
    return cudaSuccess;
  }
  cudaError_t e = cudaEventCreate(ev);
  if (e != cudaSuccess) return e;
  event_pool.push_back(*ev);
  ++event_pool_used;
  return cudaSuccess;
}

Batch Model::batch_for(const int32_t* d_slots, int32_t count) const {
  Batch b;
  b.arena = arena;
  b.slot_bytes = (int64_t)slot_bytes;
  b.slots = d_slots;
  b.counters = counters;
  b.seeds = seeds;
  b.count = count;
  return b;
}

// Splits a buffer into chains of at most max_steps steps; stages host I/O.
cc_status Model::process(const int32_t* d_slots, int32_t count, const float* in, int64_t in_stride,
                         int64_t n_in, float* out, int64_t out_stride, int64_t n_out,
                         cudaStream_t st) {
  const int32_t cin = nodes.front().d.c_in, cout = nodes.back().d.c_out;
  const int32_t ops = nodes.back().u;
  if (n_in < 0 || n_in % in_per_step != 0)
    return fail(CC_ERR_BAD_LENGTH, "n_in %lld is not a multiple of the model step (%d input frames)",
                (long long)n_in, in_per_step);
  const int64_t total_steps = n_in / in_per_step;
  if (n_out != total_steps * ops)
    return fail(CC_ERR_BAD_LENGTH, "n_out %lld != %lld steps x %d output frames", (long long)n_out,
                (long long)total_steps, ops);
  if (total_steps == 0) return CC_OK;
  if (!in || !out) return fail(CC_ERR_INVALID_ARG, "null buffer");
  const bool host_in = !is_device_ptr(in), host_out = !is_device_ptr(out);
  const Batch b = batch_for(d_slots, count);
  for (int64_t done = 0; done < total_steps; done += max_steps) {
    const int32_t steps = (int32_t)std::min<int64_t>(max_steps, total_steps - done);
    const float* cin_ptr = in + done * in_per_step * cin;
    float* cout_ptr = out + done * ops * cout;
    int64_t is = in_stride, os = out_stride;
    Staging* sg = nullptr;
    if (host_in || host_out) {
      cc_status s = ensure_staging(count, st, &sg);
      if (s) return s;
    }
    if (host_in) {
      const size_t width = (size_t)steps * in_per_step * cin * sizeof(float);
      CC_CUDA(cudaMemcpy2DAsync(sg->in, width, cin_ptr, (size_t)in_stride * sizeof(float), width,
                                count, cudaMemcpyHostToDevice, st));
      cin_ptr = sg->in;
      is = (int64_t)steps * in_per_step * cin;
    }
    float* dst = host_out ? sg->out : cout_ptr;
    if (host_out) os = (int64_t)steps * ops * cout;
    cc_status s = CC_OK;
    if (host_in && host_out && !timing_on && !force_tile_n) {
      // the chain reads and writes the staging buffers only: replay it
      cudaGraphExec_t ge = nullptr;
      for (const ChainGraph& g : chain_graphs)
        if (g.count == count && g.steps == steps && g.d_slots == d_slots && g.in == sg->in && g.out == sg->out)
          ge = g.exec;
      if (!ge) {
        if (!capture_stream) CC_CUDA(cudaStreamCreateWithFlags(&capture_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        CC_CUDA(cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal));
        s = run_chain(b, cin_ptr, is, dst, os, steps, capture_stream);
        const cudaError_t ce = cudaStreamEndCapture(capture_stream, &graph);
        if (s) {
          if (graph) cudaGraphDestroy(graph);
          return s;
        }
        if (ce != cudaSuccess) return fail(CC_ERR_CUDA, "chain capture: %s", cudaGetErrorString(ce));
        const cudaError_t ie = cudaGraphInstantiate(&ge, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return fail(CC_ERR_CUDA, "chain graph: %s", cudaGetErrorString(ie));
        chain_graphs.push_back(ChainGraph{count, steps, d_slots, sg->in, sg->out, ge});
      }
      CC_CUDA(cudaGraphLaunch(ge, st));
    } else {
      s = run_chain(b, cin_ptr, is, dst, os, steps, st);
    }
    if (s) return s;
    if (host_out) {
      const size_t width = (size_t)steps * ops * cout * sizeof(float);
      CC_CUDA(cudaMemcpy2DAsync(cout_ptr, (size_t)out_stride * sizeof(float), sg->out, width, width,
                                count, cudaMemcpyDeviceToHost, st));
    }
  }
  return CC_OK;
}

void Model::drop_chain_graphs(const float* in, const float* out) {
  // (all of them without arguments; else the ones using that staging)
  std::vector<ChainGraph> keep;
  for (auto& g : chain_graphs) {
    if (in || out) {
      if (g.in != in && g.out != out) {
        keep.push_back(g);
        continue;
      }
    }
    cudaGraphExecDestroy(g.exec);
  }
  chain_graphs.swap(keep);
}

cc_status Model::ensure_staging(int32_t count, cudaStream_t st, Staging** out) {
  const int32_t cin = nodes.front().d.c_in, cout = nodes.back().d.c_out;
  const size_t need_in = (size_t)count * max_steps * in_per_step * cin * sizeof(float);
  const size_t need_out = (size_t)count * max_steps * nodes.back().u * cout * sizeof(float);
  Staging& g = stagings[st];
  if (need_in > g.in_bytes || need_out > g.out_bytes) {
    // this stream's earlier work (and a chain replayed into them) ends first
    CC_CUDA(cudaStreamSynchronize(st));
    if (g.in || g.out) drop_chain_graphs(g.in, g.out);
  }
  if (need_in > g.in_bytes) {
    if (g.in) cudaFree(g.in);
    g.in = nullptr;
    g.in_bytes = 0;
    CC_CUDA(cudaMalloc(&g.in, need_in));
    g.in_bytes = need_in;
  }
  if (need_out > g.out_bytes) {
    if (g.out) cudaFree(g.out);
    g.out = nullptr;
    g.out_bytes = 0;
    CC_CUDA(cudaMalloc(&g.out, need_out));
    g.out_bytes = need_out;
  }
  *out = &g;
  return CC_OK;
}

Model::~Model() {
  for (auto& p : nodes) {
    if (p.dA) cudaFree(p.dA);
    if (p.dbias) cudaFree(p.dbias);
    if (p.dA_lp) cudaFree(p.dA_lp);
    if (p.dA_tiled) cudaFree(p.dA_tiled);
    if (p.dscale) cudaFree(p.dscale);
  }
  if (err) cudaFree(err);
  if (withhold) cudaFree(withhold);
  if (arena) cudaFree(arena);
  if (counters) cudaFree(counters);
  if (seeds) cudaFree(seeds);
  if (in_manip) cudaFree(in_manip);
  for (auto& kv : slot_lists) {
    if (kv.second.d) cudaFree(kv.second.d);
    if (kv.second.h) cudaFreeHost(kv.second.h);
    if (kv.second.uploaded) cudaEventDestroy(kv.second.uploaded);
  }
  drop_chain_graphs();
  if (capture_stream) cudaStreamDestroy(capture_stream);
  for (auto& kv : stagings) {
    if (kv.second.in) cudaFree(kv.second.in);
    if (kv.second.out) cudaFree(kv.second.out);
  }
  if (d_state_regions) cudaFree(d_state_regions);
  if (rag_in) cudaFree(rag_in);
  if (rag_out) cudaFree(rag_out);
  for (auto e : event_pool) cudaEventDestroy(e);
}

}  // namespace cc

// ===========================================================================
// C ABI
// ===========================================================================
using cc::fail;

namespace cc {
// Device list of the batch's slots for launches on CUDA stream `st`: one list
// per CUDA stream (batches on different streams may run concurrently),
// re-uploaded only when the slots change.  The pinned staging buffer may
// still feed the stream's previous upload, so that upload is waited for first.
cc_status upload_slot_list(Model* m, const std::vector<int32_t>& slots, cudaStream_t st, const int32_t** d_list) {
  Model::SlotList* L;
  {
    std::lock_guard<std::mutex> g(m->mu);
    L = &m->slot_lists[st];
    if (!L->d) {
      if (cudaMalloc(&L->d, sizeof(int32_t) * m->max_streams) != cudaSuccess ||
          cudaMallocHost(&L->h, sizeof(int32_t) * m->max_streams) != cudaSuccess ||
          cudaEventCreateWithFlags(&L->uploaded, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(CC_ERR_NO_MEMORY, "batch slot list");
      }
    }
  }
  if (!L->valid || L->cache != slots) {
    CC_CUDA(cudaEventSynchronize(L->uploaded));
    std::memcpy(L->h, slots.data(), sizeof(int32_t) * slots.size());
    CC_CUDA(cudaMemcpyAsync(L->d, L->h, sizeof(int32_t) * slots.size(), cudaMemcpyHostToDevice, st));
    CC_CUDA(cudaEventRecord(L->uploaded, st));
    L->cache = slots;
    L->valid = true;
  }
  *d_list = L->d;
  return CC_OK;
}

int32_t stream_slot(const cc_stream* s) { return s->slot; }
bool stream_manipulated(const cc_stream* s) { return s->manip_set; }
Model* stream_model(const cc_stream* s) { return s->model; }
}  // namespace cc

extern "C" {

const char* cc_last_error(void) { return cc::g_last_error.c_str(); }

const char* cc_status_str(cc_status s) {
  switch (s) {
    case CC_OK: return "ok";
    case CC_ERR_INVALID_ARG: return "invalid argument";
    case CC_ERR_BAD_GRAPH: return "bad graph";
    case CC_ERR_BAD_LENGTH: return "bad length";
    case CC_ERR_NO_MEMORY: return "no memory";
    case CC_ERR_CUDA: return "cuda error";
    case CC_ERR_TIMEOUT: return "timeout";
    case CC_ERR_STATE: return "bad state";
    default: return "unknown status";
  }
}

cc_status cc_model_create(const cc_node_desc* nodes, int32_t n_nodes, const float* const* weights,
                          const float* const* biases, const cc_model_config* config, cc_model** out) {
  if (!nodes || !config || !out || n_nodes <= 0) return fail(CC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (config->compute != CC_F32 && config->compute != CC_BF16 && config->compute != CC_F16)
    return fail(CC_ERR_INVALID_ARG, "unknown compute dtype %d", config->compute);
  if (config->max_streams < 0 || config->max_steps_per_call <= 0 || config->arena_bytes < 0 ||
      config->wait_limit_ns < 0)
    return fail(CC_ERR_INVALID_ARG,
                "max_streams, arena_bytes and wait_limit_ns must be >= 0 and max_steps_per_call > 0");
  auto* m = new cc::Model();
  m->dtype = config->compute;
  m->lp_dtype = config->compute == CC_F16 ? cc::kDtF16 : cc::kDtBF16;
  m->max_streams = config->max_streams;
  m->max_steps = config->max_steps_per_call;
  if (config->wait_limit_ns > 0) m->wait_ns = (uint64_t)config->wait_limit_ns;
  m->noise = config->noise ? 1 : 0;
  m->fuse_units = (config->flags & CC_FLAG_NO_UNIT_FUSION) ? 0 : 1;
  m->merge_siblings = (config->flags & CC_FLAG_NO_SIBLING_MERGE) ? 0 : 1;
  m->nodes.resize(n_nodes);
  for (int i = 0; i < n_nodes; ++i) m->nodes[i].d = nodes[i];
  cc_status s = cc::validate_and_analyze(*m);
  if (!s) {
    cc::plan_fusion(*m);
    cc::plan_siblings(*m);
    s = cc::plan_arena(*m);
  }
  if (!s && config->arena_bytes > 0) {
    // admission by cache memory: as many slots as the byte budget holds
    const int64_t fit = config->arena_bytes / (int64_t)m->slot_bytes;
    int64_t slots = config->max_streams > 0 ? std::min<int64_t>(fit, config->max_streams) : fit;
    slots = std::min<int64_t>(slots, INT32_MAX);
    if (slots < 1)
      s = fail(CC_ERR_NO_MEMORY, "arena budget of %lld bytes holds no stream slot (%zu bytes each)",
               (long long)config->arena_bytes, m->slot_bytes);
    else
      m->max_streams = (int32_t)slots;
  }
  if (!s && m->max_streams == 0) {  // plan only: analysis queries, no device memory
    *out = reinterpret_cast<cc_model*>(m);
    return CC_OK;
  }
  if (!s) s = cc::pack_and_upload(*m, weights, biases);
  if (!s) {
    cc::plan_units(*m);
    cc::plan_ksplit(*m);
  }
  if (!s) {
    const size_t arena_bytes = m->slot_bytes * (size_t)m->max_streams;
    // the tensor-core epilogue addresses the arena in 32-bit 16-byte units
    cudaError_t e = arena_bytes >= (size_t(1) << 36) ? cudaErrorMemoryAllocation
                                                     : cudaMalloc(&m->arena, arena_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      m->arena = nullptr;
      s = fail(CC_ERR_NO_MEMORY, "arena of %zu bytes: %s", arena_bytes, cudaGetErrorString(e));
    }
  }
  if (!s) s = cc::encode_gather_maps(*m);
  if (!s) s = cc::plan_state(*m);
  if (!s && !m->state_regions.empty()) {
    const size_t nb = sizeof(cc::Model::StateRegion) * m->state_regions.size();
    if (cudaMalloc(&m->d_state_regions, nb) != cudaSuccess ||
        cudaMemcpy(m->d_state_regions, m->state_regions.data(), nb, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      s = fail(CC_ERR_NO_MEMORY, "state map");
    }
  }
  const size_t manip_floats = (size_t)3 * m->nodes.front().d.c_out * m->max_streams;
  if (!s && (cudaMalloc(&m->counters, sizeof(int64_t) * m->max_streams) != cudaSuccess ||
             cudaMalloc(&m->seeds, sizeof(uint64_t) * m->max_streams) != cudaSuccess ||
             cudaMalloc(&m->in_manip, sizeof(float) * manip_floats) != cudaSuccess ||

             cudaMalloc(&m->err, sizeof(int32_t)) != cudaSuccess ||
             cudaMalloc(&m->withhold, sizeof(int32_t)) != cudaSuccess))
    s = fail(CC_ERR_NO_MEMORY, "model bookkeeping allocation failed");
  if (!s && (cudaMemset(m->counters, 0, sizeof(int64_t) * m->max_streams) != cudaSuccess ||
             cudaMemset(m->err, 0, sizeof(int32_t)) != cudaSuccess ||
             cudaMemset(m->withhold, 0, sizeof(int32_t)) != cudaSuccess ||
             cudaMemset(m->seeds, 0, sizeof(uint64_t) * m->max_streams) != cudaSuccess))
    s = fail(CC_ERR_CUDA, "memset failed");
  if (!s) {  // every slot starts with the identity input manipulation
    const int32_t C = m->nodes.front().d.c_out;
    std::vector<float> ident(manip_floats, 0.f);
    for (int32_t slot = 0; slot < m->max_streams; ++slot)
      std::fill_n(ident.begin() + (size_t)slot * 3 * C, C, 1.f);
    if (cudaMemcpy(m->in_manip, ident.data(), sizeof(float) * manip_floats, cudaMemcpyHostToDevice) !=
        cudaSuccess)
      s = fail(CC_ERR_CUDA, "input manipulation upload failed");
  }
  if (s) {
    delete m;
    return s;
  }
  for (int i = m->max_streams - 1; i >= 0; --i) m->free_slots.push_back(i);
  *out = reinterpret_cast<cc_model*>(m);
  return CC_OK;
}

cc_status cc_model_destroy(cc_model* model) {
  if (!model) return fail(CC_ERR_INVALID_ARG, "null model");
  auto* m = reinterpret_cast<cc::Model*>(model);
  if (m->max_streams > 0) cudaDeviceSynchronize();
  for (cc_stream* s : m->live_streams) {  // streams die with their model
    if (s->d_slot) cudaFree(s->d_slot);
    cc::free_fifo(s);
    delete s;
  }
  m->live_streams.clear();
  delete m;
  return CC_OK;
}

cc_status cc_model_total_delay(const cc_model* model, int64_t* out_frames) {
  if (!model || !out_frames) return fail(CC_ERR_INVALID_ARG, "null argument");
  *out_frames = reinterpret_cast<const cc::Model*>(model)->nodes.back().D;
  return CC_OK;
}

cc_status cc_model_io(const cc_model* model, int32_t* in_ch, int32_t* out_ch, int32_t* in_per_step,
                      int32_t* out_per_step) {
  if (!model) return fail(CC_ERR_INVALID_ARG, "null model");
  auto* m = reinterpret_cast<const cc::Model*>(model);
  if (in_ch) *in_ch = m->nodes.front().d.c_in;
  if (out_ch) *out_ch = m->nodes.back().d.c_out;
  if (in_per_step) *in_per_step = m->in_per_step;
  if (out_per_step) *out_per_step = m->nodes.back().u;
  return CC_OK;
}

cc_status cc_model_node_info(const cc_model* model, int32_t node, int64_t* delay, int32_t* extra_delay,
                             int32_t* align3, int32_t* kept, int32_t* fps) {
  if (!model) return fail(CC_ERR_INVALID_ARG, "null model");
  auto* m = reinterpret_cast<const cc::Model*>(model);
  if (node < 0 || node >= (int)m->nodes.size()) return fail(CC_ERR_INVALID_ARG, "node %d out of range", node);
  const auto& p = m->nodes[node];
  if (delay) *delay = p.D;
  if (extra_delay) *extra_delay = p.Da;
  if (align3)
    for (int q = 0; q < 3; ++q) align3[q] = p.A[q];
  if (kept) *kept = p.keep;
  if (fps) *fps = p.u;
  return CC_OK;
}

cc_status cc_model_capacity(const cc_model* model, int32_t* max_streams, int32_t* free_slots) {
  if (!model) return fail(CC_ERR_INVALID_ARG, "null model");
  auto* m = const_cast<cc::Model*>(reinterpret_cast<const cc::Model*>(model));
  std::lock_guard<std::mutex> g(m->mu);
  if (max_streams) *max_streams = m->max_streams;
  if (free_slots) *free_slots = (int32_t)m->free_slots.size();
  return CC_OK;
}

cc_status cc_model_state_bytes(const cc_model* model, size_t* state_bytes, size_t* slot_bytes) {
  if (!model) return fail(CC_ERR_INVALID_ARG, "null model");
  auto* m = reinterpret_cast<const cc::Model*>(model);
  if (state_bytes) *state_bytes = m->state_bytes;
  if (slot_bytes) *slot_bytes = m->slot_bytes;
  return CC_OK;
}

// Uploads one slot's input manipulation (scale, bias, noise amplitude: host,
// [C] each; NULL means 1 / 0 / 0) on `st` and waits for it.
static cc_status upload_manip(cc::Model* m, int32_t slot, const float* scale, const float* bias,
                              const float* noise, cudaStream_t st) {
  const int32_t C = m->nodes.front().d.c_out;
  std::vector<float> rows(3 * (size_t)C);
  for (int32_t c = 0; c < C; ++c) {
    rows[c] = scale ? scale[c] : 1.f;
    rows[C + c] = bias ? bias[c] : 0.f;
    rows[2 * C + c] = noise ? noise[c] : 0.f;
  }
  CC_CUDA(cudaMemcpyAsync(m->in_manip + (size_t)slot * 3 * C, rows.data(), sizeof(float) * rows.size(),
                          cudaMemcpyHostToDevice, st));
  CC_CUDA(cudaStreamSynchronize(st));  // rows leave scope on return
  return CC_OK;
}

static cc_status zero_slot(cc::Model* m, int32_t slot, uint64_t seed, cudaStream_t st) {
  CC_CUDA(cudaMemsetAsync(m->arena + (size_t)slot * m->slot_bytes, 0, m->slot_bytes, st));
  CC_CUDA(cudaMemsetAsync(m->counters + slot, 0, sizeof(int64_t), st));
  const uint64_t host_seed = seed;
  CC_CUDA(cudaMemcpyAsync(m->seeds + slot, &host_seed, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  CC_CUDA(cudaStreamSynchronize(st));  // host_seed leaves scope on return
  return upload_manip(m, slot, nullptr, nullptr, nullptr, st);
}

cc_status cc_stream_create(cc_model* model, uint64_t seed, void* cuda_stream, cc_stream** out) {
  if (!model || !out) return fail(CC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  auto* m = reinterpret_cast<cc::Model*>(model);
  int32_t slot;
  {
    std::lock_guard<std::mutex> g(m->mu);
    if (m->free_slots.empty())
      return fail(CC_ERR_NO_MEMORY, "arena full: all %d stream slots (%zu bytes each) are in use",
                  m->max_streams, m->slot_bytes);
    slot = m->free_slots.back();
    m->free_slots.pop_back();
  }
  auto* s = new cc_stream{m, slot, seed, nullptr};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  cc_status r = CC_OK;
  if (cudaMalloc(&s->d_slot, sizeof(int32_t)) != cudaSuccess) {
    r = fail(CC_ERR_NO_MEMORY, "stream handle allocation failed");
  } else if (cudaMemcpy(s->d_slot, &slot, sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    r = fail(CC_ERR_CUDA, "stream handle upload failed");
  } else {
    r = zero_slot(m, slot, seed, st);
  }
  if (r) {
    if (s->d_slot) cudaFree(s->d_slot);
    std::lock_guard<std::mutex> g(m->mu);
    m->free_slots.push_back(slot);
    delete s;
    return r;
  }
  {
    std::lock_guard<std::mutex> g(m->mu);
    m->live_streams.push_back(s);
  }
  *out = s;
  return CC_OK;
}

cc_status cc_stream_destroy(cc_stream* s) {
  if (!s) return fail(CC_ERR_INVALID_ARG, "null stream");
  cudaDeviceSynchronize();
  cudaFree(s->d_slot);
  cc::free_fifo(s);
  {
    cc::Model* m = s->model;
    std::lock_guard<std::mutex> g(m->mu);
    m->free_slots.push_back(s->slot);
    for (auto& kv : m->slot_lists) kv.second.valid = false;
    m->live_streams.erase(std::remove(m->live_streams.begin(), m->live_streams.end(), s),
                          m->live_streams.end());
  }
  delete s;
  return CC_OK;
}

cc_status cc_stream_reset(cc_stream* s, void* cuda_stream) {
  if (!s) return fail(CC_ERR_INVALID_ARG, "null stream");
  s->manip_set = false;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (s->fifo) {  // back to the state FIFO mode started in: no pending input, the prefill queued
    const int32_t cout = s->model->nodes.back().d.c_out;
    s->in_frames = 0;
    s->out_cur = 0;
    s->out_frames = s->prefill;
    if (s->prefill) CC_CUDA(cudaMemsetAsync(s->out_q[0], 0, sizeof(float) * s->prefill * cout, st));
  }
  return zero_slot(s->model, s->slot, s->seed, st);
}

cc_status cc_stream_set_input_manipulation(cc_stream* s, const float* scale, const float* bias,
                                           const float* noise, int32_t channels, void* cuda_stream) {
  if (!s) return fail(CC_ERR_INVALID_ARG, "null stream");
  cc::Model* m = s->model;
  const int32_t C = m->nodes.front().d.c_out;
  if (channels != C) return fail(CC_ERR_INVALID_ARG, "channels %d != the model's %d input channels", channels, C);
  bool ident = true;
  for (int32_t c = 0; c < C; ++c) {
    const float a = scale ? scale[c] : 1.f, b = bias ? bias[c] : 0.f, q = noise ? noise[c] : 0.f;
    if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(q))
      return fail(CC_ERR_INVALID_ARG, "non-finite value at channel %d", c);
    ident = ident && a == 1.f && b == 0.f && q == 0.f;
  }
  const cc_status r = upload_manip(m, s->slot, scale, bias, noise, reinterpret_cast<cudaStream_t>(cuda_stream));
  if (!r) s->manip_set = !ident;
  return r;
}

cc_status cc_stream_process(cc_stream* s, const float* in, int64_t n_in, float* out, int64_t n_out,
                            void* cuda_stream) {
  if (!s) return fail(CC_ERR_INVALID_ARG, "null stream");
  cc::Model* m = s->model;
  if (s->fifo) return cc::process_ragged(m, &s, &in, &n_in, &out, &n_out, 1, reinterpret_cast<cudaStream_t>(cuda_stream));
  const int32_t cin = m->nodes.front().d.c_in, cout = m->nodes.back().d.c_out;
  return m->process(s->d_slot, 1, in, n_in * cin, n_in, out, n_out * cout, n_out,
                    reinterpret_cast<cudaStream_t>(cuda_stream));
}

cc_status cc_process_batch_strided(cc_model* model, cc_stream* const* streams, int32_t count, const float* in,
                                   int64_t in_stride, int64_t n_in, float* out, int64_t out_stride, int64_t n_out,
                                   void* cuda_stream) {
  if (!model || !streams || count <= 0) return fail(CC_ERR_INVALID_ARG, "null argument or empty batch");
  auto* m = reinterpret_cast<cc::Model*>(model);
  if (count > m->max_streams) return fail(CC_ERR_INVALID_ARG, "batch larger than max_streams");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  std::vector<int32_t> slots(count);
  for (int i = 0; i < count; ++i) {
    if (!streams[i] || streams[i]->model != m) return fail(CC_ERR_INVALID_ARG, "stream %d not of this model", i);
    if (streams[i]->fifo)
      return fail(CC_ERR_STATE, "stream %d is in FIFO mode: use cc_process_batch or cc_stream_process", i);
    slots[i] = streams[i]->slot;
  }
  {
    std::vector<int32_t> sorted = slots;
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(CC_ERR_INVALID_ARG, "a stream appears twice in one batch");
  }
  const int32_t* d_list = nullptr;
  cc_status r = cc::upload_slot_list(m, slots, st, &d_list);
  if (r) return r;
  return m->process(d_list, count, in, in_stride, n_in, out, out_stride, n_out, st);
}

cc_status cc_process_batch(cc_model* model, cc_stream* const* streams, const float* const* in,
                           const int64_t* n_in, float* const* out, const int64_t* n_out, int32_t count,
                           void* cuda_stream) {
  if (!model || !streams || !n_in || !n_out || count <= 0)
    return fail(CC_ERR_INVALID_ARG, "null argument or empty batch");
  auto* m = reinterpret_cast<cc::Model*>(model);
  return cc::process_ragged(m, streams, in, n_in, out, n_out, count, reinterpret_cast<cudaStream_t>(cuda_stream));
}

cc_status cc_stream_state_size(const cc_stream* s, size_t* bytes) {
  if (!s || !bytes) return fail(CC_ERR_INVALID_ARG, "null argument");
  *bytes = s->model->slot_bytes + 2 * sizeof(uint64_t);
  return CC_OK;
}

cc_status cc_stream_get_state(cc_stream* s, void* blob, size_t bytes, void* cuda_stream) {
  if (!s || !blob) return fail(CC_ERR_INVALID_ARG, "null argument");
  cc::Model* m = s->model;
  if (bytes != m->slot_bytes + 2 * sizeof(uint64_t)) return fail(CC_ERR_INVALID_ARG, "state blob size mismatch");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  auto* b = static_cast<char*>(blob);
  CC_CUDA(cudaMemcpyAsync(b, m->counters + s->slot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CC_CUDA(cudaMemcpyAsync(b + 8, m->seeds + s->slot, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  CC_CUDA(cudaMemcpyAsync(b + 16, m->arena + (size_t)s->slot * m->slot_bytes, m->slot_bytes,
                          cudaMemcpyDeviceToHost, st));
  CC_CUDA(cudaStreamSynchronize(st));
  return CC_OK;
}

cc_status cc_stream_set_state(cc_stream* s, const void* blob, size_t bytes, void* cuda_stream) {
  if (!s || !blob) return fail(CC_ERR_INVALID_ARG, "null argument");
  cc::Model* m = s->model;
  if (bytes != m->slot_bytes + 2 * sizeof(uint64_t)) return fail(CC_ERR_INVALID_ARG, "state blob size mismatch");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  auto* b = static_cast<const char*>(blob);
  CC_CUDA(cudaMemcpyAsync(m->counters + s->slot, b, sizeof(int64_t), cudaMemcpyHostToDevice, st));
  CC_CUDA(cudaMemcpyAsync(m->seeds + s->slot, b + 8, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  CC_CUDA(cudaMemcpyAsync(m->arena + (size_t)s->slot * m->slot_bytes, b + 16, m->slot_bytes,
                          cudaMemcpyHostToDevice, st));
  CC_CUDA(cudaStreamSynchronize(st));
  std::memcpy(&s->seed, b + 8, sizeof(uint64_t));
  return CC_OK;
}

cc_status cc_model_device_status(cc_model* model, int32_t* code) {
  if (!model) return fail(CC_ERR_INVALID_ARG, "null model");
  auto* m = reinterpret_cast<cc::Model*>(model);
  int32_t v = 0;
  if (m->err) {
    CC_CUDA(cudaDeviceSynchronize());
    CC_CUDA(cudaMemcpy(&v, m->err, sizeof(int32_t), cudaMemcpyDeviceToHost));
    CC_CUDA(cudaMemset(m->err, 0, sizeof(int32_t)));
  }
  if (code) *code = v;
  if (v) return fail(CC_ERR_TIMEOUT, "a bounded device wait gave up (code %d)", v);
  return CC_OK;
}

cc_status cc_model_test_withhold_copy(cc_model* model, int32_t launches) {
  if (!model || launches < 0) return fail(CC_ERR_INVALID_ARG, "null model or negative count");
  auto* m = reinterpret_cast<cc::Model*>(model);
  if (!m->withhold) return fail(CC_ERR_STATE, "a plan-only model launches nothing");
  CC_CUDA(cudaDeviceSynchronize());
  CC_CUDA(cudaMemcpy(m->withhold, &launches, sizeof(int32_t), cudaMemcpyHostToDevice));
  return CC_OK;
}

cc_status cc_model_chain_launches(const cc_model* model, int32_t* launches) {
  if (!model || !launches) return fail(CC_ERR_INVALID_ARG, "null argument");
  *launches = reinterpret_cast<const cc::Model*>(model)->last_chain_launches;
  return CC_OK;
}

cc_status cc_model_timing(cc_model* model, int32_t enable) {
  if (!model) return fail(CC_ERR_INVALID_ARG, "null model");
  auto* m = reinterpret_cast<cc::Model*>(model);
  CC_CUDA(cudaDeviceSynchronize());
  m->timing_on = enable != 0;
  m->timing_recs.clear();
  m->event_pool_used = 0;
  return CC_OK;
}

cc_status cc_model_timing_read(cc_model* model, double* ms, int64_t* launches, int32_t n_nodes) {
  if (!model) return fail(CC_ERR_INVALID_ARG, "null model");
  auto* m = reinterpret_cast<cc::Model*>(model);
  if (n_nodes != (int)m->nodes.size()) return fail(CC_ERR_INVALID_ARG, "n_nodes mismatch");
  for (int i = 0; i < n_nodes; ++i) {
    if (ms) ms[i] = 0.0;
    if (launches) launches[i] = 0;
  }
  for (auto& r : m->timing_recs) {
    CC_CUDA(cudaEventSynchronize(r.stop));
    float t = 0.f;
    CC_CUDA(cudaEventElapsedTime(&t, r.start, r.stop));
    if (ms) ms[r.node] += t;
    if (launches) launches[r.node] += 1;
  }
  return CC_OK;
}

}  // extern "C"
