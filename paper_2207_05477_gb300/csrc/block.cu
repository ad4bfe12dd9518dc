// Evoformer block drivers: the AlphaFold2 Algorithm 6 order of sub-modules,
// each a short chain of libevo kernels, forward (optionally keeping every
// intermediate for the backward) and backward with per-block recompute
// (HelixFold keeps only block inputs and recomputes the rest, Sec. 3.4.1).
//
// One driver serves both storage types: act_dtype EVO_BF16 runs the tcgen05
// GEMMs and tensor-core attention, EVO_F32 the plain SIMT kernels.  Weights
// enter the GEMMs straight from the flat parameter buffer (or its BF16 copy):
// a forward projection uses W [out,in] as a K-major operand and the backward
// dX = dY W uses the same buffer as an MN-major operand, so no transposed
// copies exist.  Residual-stream gradients accumulate in FP32.
#include <cmath>
#include <algorithm>
#include <map>

#include "block.h"

namespace evo {

// ------------------------------------------------------------ param table
int64_t build_param_table(const evo_dims &d, std::vector<PEntry> &out, bool pair_only) {
  out.clear();
  int64_t off = 0;
  auto add = [&](const std::string &name, std::initializer_list<int64_t> shape) {
    PEntry e;
    e.name = name;
    e.offset = off;
    e.ndim = (int)shape.size();
    int64_t n = 1;
    int k = 0;
    for (int64_t v : shape) {
      e.shape[k++] = v;
      n *= v;
    }
    for (; k < 4; ++k) e.shape[k] = 0;
    out.push_back(e);
    off += (n + 63) / 64 * 64;
  };
  auto ln = [&](const std::string &p, int64_t c) {
    add(p + ".gamma", {c});
    add(p + ".beta", {c});
  };
  const int64_t C = d.c_m, Z = d.c_z, hm = d.h_msa, cm = d.c_msa, ht = d.h_tri, ct = d.c_tri;
  if (!pair_only) {
  ln("row.ln_m", C);
  ln("row.ln_z", Z);
  add("row.w_b", {hm, Z});
  add("row.w_qkvg", {4 * hm * cm, C});
  add("row.b_g", {hm * cm});
  add("row.w_o", {C, hm * cm});
  add("row.b_o", {C});
  ln("col.ln", C);
  if (d.msa_col_mode == EVO_COL_ATTENTION) add("col.w_qkvg", {4 * hm * cm, C});
  else add("col.w_qkvg", {2 * hm * cm + 2 * cm, C});
  add("col.b_g", {hm * cm});
  add("col.w_o", {C, hm * cm});
  add("col.b_o", {C});
  ln("msa_trans.ln", C);
  add("msa_trans.w1", {d.trans_n * C, C});
  add("msa_trans.b1", {d.trans_n * C});
  add("msa_trans.w2", {C, d.trans_n * C});
  add("msa_trans.b2", {C});
  ln("opm.ln", C);
  add("opm.w_ab", {2 * d.c_opm, C});
  add("opm.b_ab", {2 * d.c_opm});
  add("opm.w_o", {Z, (int64_t)d.c_opm * d.c_opm});
  add("opm.b_o", {Z});
  }
  // the pair stack (shared by the Evoformer and the template pair block)
  for (const char *t : {"tri_out", "tri_in"}) {
    const std::string p(t);
    ln(p + ".ln_in", Z);
    add(p + ".w_abg", {4 * d.c_mul + Z, Z});
    add(p + ".b_abg", {4 * d.c_mul + Z});
    ln(p + ".ln_out", d.c_mul);
    add(p + ".w_o", {Z, d.c_mul});
    add(p + ".b_o", {Z});
  }
  for (const char *t : {"att_start", "att_end"}) {
    const std::string p(t);
    ln(p + ".ln", Z);
    add(p + ".w_b", {ht, Z});
    add(p + ".w_qkvg", {4 * ht * ct, Z});
    add(p + ".b_g", {ht * ct});
    add(p + ".w_o", {Z, ht * ct});
    add(p + ".b_o", {Z});
  }
  ln("pair_trans.ln", Z);
  add("pair_trans.w1", {d.trans_n * Z, Z});
  add("pair_trans.b1", {d.trans_n * Z});
  add("pair_trans.w2", {Z, d.trans_n * Z});
  add("pair_trans.b2", {Z});
  return off;
}

int validate_pair_dims(const evo_dims *d) {
  if (!d) return EVO_ERR_INVALID_ARG;
  if (d->n_res <= 0 || d->c_z <= 0 || d->h_tri <= 0 || d->c_tri <= 0 || d->c_mul <= 0 || d->trans_n <= 0)
    return EVO_ERR_INVALID_ARG;
  if (d->act_dtype != EVO_F32 && d->act_dtype != EVO_BF16) return EVO_ERR_INVALID_ARG;
  if (d->c_z % 8 || d->c_mul % 8 || d->c_tri % 8) return EVO_ERR_UNSUPPORTED;
  if (d->h_tri > 8 || d->c_tri > 32 || d->c_z > 1024 || d->c_mul > 256) return EVO_ERR_UNSUPPORTED;
  return EVO_OK;
}

int validate_dims(const evo_dims *d) {
  if (!d) return EVO_ERR_INVALID_ARG;
  if (d->n_seq <= 0 || d->n_res <= 0 || d->c_m <= 0 || d->c_z <= 0 || d->h_msa <= 0 || d->c_msa <= 0 ||
      d->h_tri <= 0 || d->c_tri <= 0 || d->c_mul <= 0 || d->c_opm <= 0 || d->trans_n <= 0)
    return EVO_ERR_INVALID_ARG;
  if (d->act_dtype != EVO_F32 && d->act_dtype != EVO_BF16) return EVO_ERR_INVALID_ARG;
  if (d->msa_col_mode != EVO_COL_ATTENTION && d->msa_col_mode != EVO_COL_GLOBAL) return EVO_ERR_INVALID_ARG;
  // kernels: channel dims multiples of 8 (16-byte rows), heads <= 8, head dim <= 32
  if (d->c_m % 8 || d->c_z % 8 || d->c_mul % 8 || d->c_opm % 8 || d->c_msa % 8 || d->c_tri % 8) return EVO_ERR_UNSUPPORTED;
  if (d->h_msa > 8 || d->h_tri > 8 || d->c_msa > 32 || d->c_tri > 32) return EVO_ERR_UNSUPPORTED;
  if (d->c_m > 1024 || d->c_z > 1024 || d->c_mul > 256) return EVO_ERR_UNSUPPORTED;
  if (d->msa_col_mode == EVO_COL_GLOBAL &&
      (!global_attn_supported(d->h_msa, d->c_msa) || (int64_t)d->n_seq * d->h_msa * 4 > 200 * 1024))
    return EVO_ERR_UNSUPPORTED;
  if (d->pair_slab < 0) return EVO_ERR_INVALID_ARG;
  return EVO_OK;
}

bool pair_slabbed(const evo_dims &d) { return d.pair_slab > 0 && d.pair_slab < d.n_res; }

int validate_infer_dims(const evo_dims *d) {
  const int v = validate_dims(d);
  if (v != EVO_OK || !pair_slabbed(*d)) return v;
  // the slab steps run on the BF16 TMA kernels only (pair bias projection
  // with c_z = 128 and 4 or 8 heads, channel-major gate and LayerNorm)
  const bool heads = (d->h_msa == 4 || d->h_msa == 8) && (d->h_tri == 4 || d->h_tri == 8);
  if (d->act_dtype != EVO_BF16 || d->c_z != 128 || !heads || (d->c_mul != 64 && d->c_mul != 128 && d->c_mul != 256))
    return EVO_ERR_UNSUPPORTED;
  return EVO_OK;
}

// ------------------------------------------------------------ workspace plan
namespace {

constexpr int MAXSPLIT = 32;

struct TriBufs {
  size_t xz, abg, A, B, X, xo, y, zout;
};
struct AttBufs {
  size_t xz, bias, qkvg, oatt, og, lse, zout;
};

struct Plan {
  size_t xm1, xz1, bias1, qkvg1, oatt1, og1, lse1, m1;
  size_t xm2, qkvg2, oatt2, og2, lse2, m2;
  size_t gq, gob, gst;  // global column attention: masked-mean query, output, softmax stats
  size_t xm3, h3, m3;
  size_t xm4, ab4, O4, inv4, z1;
  TriBufs tri[2];
  AttBufs att[2];
  size_t xz9, h9, z6;
  size_t dm_acc, dmT, dz_acc, dzT, G1, G2, G3, dO4, dA, dB, dX, dq_acc, dbias, Dsum, dab4, split;
  size_t drop_u;  // training-mode dropout: the update before its scale (forward), the scaled gradient (backward)
  int64_t wmax = 0;  // split holds MAXSPLIT * wmax floats
  // i-slab subbatching of the inference plan (d.pair_slab rows per slab)
  struct Slab {
    bool on = false;
    int64_t Ri = 0;                   // pair rows per slab
    size_t xz1, O4;                   // row-attention pair LayerNorm, outer products (one slab)
    size_t zT, pmT;                   // full-size: transposed z and pair mask (incoming, ending)
    size_t Bfull;                     // full-size: channel-major b of a triangle product
    size_t xz, abg, A, X, xo, y;      // triangle multiplication (one slab)
    size_t tbias;                     // full-size: triangle attention pair bias
    size_t axz, qkvg, oatt, og, lse;  // triangle attention (one slab)
    size_t txz, h;                    // pair transition (one slab)
  } sl;
  size_t total;
};

struct Dims2 {
  int64_t S, R, Cm, Cz, Hm, cm, Ht, ct, cmul, co, n, Mm, Mz, Rp, HCm, HCt, QKm, QKc, ABG;
  // pair_only: the template pair block, no MSA (every MSA size 0)
  explicit Dims2(const evo_dims &d, bool pair_only = false) {
    S = pair_only ? 0 : d.n_seq, R = d.n_res, Cm = d.c_m, Cz = d.c_z, Hm = d.h_msa, cm = d.c_msa, Ht = d.h_tri, ct = d.c_tri;
    cmul = d.c_mul, co = d.c_opm, n = d.trans_n;
    Mm = S * R, Mz = R * R, Rp = (R + 7) / 8 * 8;
    HCm = Hm * cm, HCt = Ht * ct;
    QKm = 4 * HCm;
    QKc = d.msa_col_mode == EVO_COL_ATTENTION ? 4 * HCm : 2 * HCm + 2 * cm;
    ABG = 4 * cmul + Cz;
  }
};

// Forward-only plan (inference; no backward reads the intermediates).  Once a
// sub-module has written its output nothing else of it is read again, so the
// scratch of every sub-module starts at one common offset, and the residual
// streams alternate between two buffers each: m1, m2, then m3 over m1; z1 and
// a second buffer, the five pair updates writing them in turn.  Every buffer
// keeps the size it has in the full plan.
size_t make_infer_plan(const evo_dims &d, Plan &p, bool pair_only) {
  const Dims2 k(d, pair_only);
  const size_t ts = d.act_dtype == EVO_BF16 ? 2 : 4;
  p = Plan{};
  size_t off = 0, top = 0;
  auto T = [&](int64_t elems) {
    size_t o = off;
    off += ((size_t)elems * ts + 255) / 256 * 256;
    return o;
  };
  auto F = [&](int64_t elems) {
    size_t o = off;
    off += ((size_t)elems * 4 + 255) / 256 * 256;
    return o;
  };
  p.m1 = T(k.Mm * k.Cm), p.m2 = T(k.Mm * k.Cm), p.m3 = p.m1;
  p.z1 = T(k.Mz * k.Cz);
  const size_t zb = T(k.Mz * k.Cz);
  p.tri[0].zout = zb, p.tri[1].zout = p.z1, p.att[0].zout = zb, p.att[1].zout = p.z1, p.z6 = zb;
  const size_t scr = off;
  p.drop_u = scr;  // evaluation only: no dropout
  auto begin = [&] { off = scr; };
  auto end = [&] { top = std::max(top, off); };
  if (!pair_only && pair_slabbed(d)) {
    // i-slab subbatching (Sec. 3.4.4): every pair-sized intermediate lives for
    // one slab of Ri pair rows only; what stays full-size is z (two buffers),
    // the channel-major b of a triangle product, the transposed z and pair
    // mask of the incoming / ending steps and the pair biases
    Plan::Slab &sl = p.sl;
    sl.on = true;
    sl.Ri = d.pair_slab;
    const int64_t Ps = sl.Ri * k.R;  // positions of a slab
    begin();  // 1. MSA row attention (the pair bias from LayerNorm(z) slab by slab)
    p.xm1 = T(k.Mm * k.Cm), sl.xz1 = T(Ps * k.Cz), p.bias1 = F(k.Hm * k.Mz), p.qkvg1 = T(k.Mm * k.QKm);
    p.oatt1 = T(k.Mm * k.HCm), p.og1 = T(k.Mm * k.HCm), p.lse1 = F(k.S * k.Hm * k.R);
    end();
    begin();  // 2. MSA column attention (or global column attention)
    p.xm2 = T(k.Mm * k.Cm), p.qkvg2 = T(k.Mm * k.QKc), p.oatt2 = T(k.Mm * k.HCm), p.og2 = T(k.Mm * k.HCm);
    p.lse2 = F(k.R * k.Hm * k.S), p.gq = F(k.R * k.HCm), p.gob = F(k.R * k.HCm), p.gst = F(k.R * k.Hm * 2);
    end();
    begin();  // 3. MSA transition
    p.xm3 = T(k.Mm * k.Cm), p.h3 = T(k.Mm * k.n * k.Cm);
    end();
    begin();  // 4. outer product mean: the outer products of one slab of rows i
    p.xm4 = T(k.Mm * k.Cm), p.ab4 = T(2 * k.Mm * k.co), p.inv4 = F(k.Mz), sl.O4 = T(Ps * k.co * k.co);
    end();
    begin();  // 5-9: the transposed z and mask live through the four triangle steps
    sl.zT = T(k.Mz * k.Cz), sl.pmT = F(k.Mz);
    const size_t pair = off;
    sl.Bfull = T(k.cmul * k.R * k.Rp);  // 5, 6. triangle multiplications
    sl.xz = T(Ps * k.Cz), sl.abg = T(Ps * k.ABG), sl.A = T(k.cmul * sl.Ri * k.Rp), sl.X = T(k.cmul * sl.Ri * k.Rp);
    sl.xo = T(Ps * k.cmul), sl.y = T(Ps * k.Cz);
    end();
    off = pair;  // 7, 8. triangle attentions
    sl.tbias = T(k.Ht * k.Mz), sl.axz = T(Ps * k.Cz), sl.qkvg = T(Ps * 4 * k.HCt), sl.oatt = T(Ps * k.HCt);
    sl.og = T(Ps * k.HCt), sl.lse = F(sl.Ri * k.Ht * k.R);
    end();
    begin();  // 9. pair transition
    sl.txz = T(Ps * k.Cz), sl.h = T(Ps * k.n * k.Cz);
    end();
    p.total = top;
    return top;
  }
  begin();  // 1. MSA row attention
  p.xm1 = T(k.Mm * k.Cm), p.xz1 = T(k.Mz * k.Cz), p.bias1 = F(k.Hm * k.Mz), p.qkvg1 = T(k.Mm * k.QKm);
  p.oatt1 = T(k.Mm * k.HCm), p.og1 = T(k.Mm * k.HCm), p.lse1 = F(k.S * k.Hm * k.R);
  end();
  begin();  // 2. MSA column attention (or global column attention)
  p.xm2 = T(k.Mm * k.Cm), p.qkvg2 = T(k.Mm * k.QKc), p.oatt2 = T(k.Mm * k.HCm), p.og2 = T(k.Mm * k.HCm);
  p.lse2 = F(k.R * k.Hm * k.S), p.gq = F(k.R * k.HCm), p.gob = F(k.R * k.HCm), p.gst = F(k.R * k.Hm * 2);
  end();
  begin();  // 3. MSA transition
  p.xm3 = T(k.Mm * k.Cm), p.h3 = T(k.Mm * k.n * k.Cm);
  end();
  const int64_t Mz_opm = pair_only ? 0 : k.Mz;
  begin();  // 4. outer product mean
  p.xm4 = T(k.Mm * k.Cm), p.ab4 = T(2 * k.Mm * k.co), p.O4 = T(Mz_opm * k.co * k.co), p.inv4 = F(Mz_opm);
  end();
  for (int t = 0; t < 2; ++t) {  // 5, 6. triangle multiplications
    TriBufs &b = p.tri[t];
    begin();
    b.xz = T(k.Mz * k.Cz), b.abg = T(k.Mz * k.ABG), b.A = T(k.cmul * k.R * k.Rp), b.B = T(k.cmul * k.R * k.Rp);
    b.X = T(k.cmul * k.R * k.Rp), b.xo = T(k.Mz * k.cmul), b.y = T(k.Mz * k.Cz);
    end();
  }
  for (int t = 0; t < 2; ++t) {  // 7, 8. triangle attentions
    AttBufs &b = p.att[t];
    begin();
    b.xz = T(k.Mz * k.Cz), b.bias = F(k.Ht * k.Mz), b.qkvg = T(k.Mz * 4 * k.HCt), b.oatt = T(k.Mz * k.HCt);
    b.og = T(k.Mz * k.HCt), b.lse = F(k.R * k.Ht * k.R);
    end();
  }
  begin();  // 9. pair transition
  p.xz9 = T(k.Mz * k.Cz), p.h9 = T(k.Mz * k.n * k.Cz);
  end();
  p.total = top;
  return top;
}

size_t make_plan(const evo_dims &d, int mode, Plan &p, bool pair_only = false) {
  if (mode == EVO_MODE_INFER) return make_infer_plan(d, p, pair_only);
  const Dims2 k(d, pair_only);
  const size_t ts = d.act_dtype == EVO_BF16 ? 2 : 4;
  size_t off = 0;
  auto T = [&](int64_t elems) {
    size_t o = off;
    off += ((size_t)elems * ts + 255) / 256 * 256;
    return o;
  };
  auto F = [&](int64_t elems) {
    size_t o = off;
    off += ((size_t)elems * 4 + 255) / 256 * 256;
    return o;
  };
  p.xm1 = T(k.Mm * k.Cm), p.xz1 = T(k.Mz * k.Cz), p.bias1 = F(k.Hm * k.Mz), p.qkvg1 = T(k.Mm * k.QKm);
  p.oatt1 = T(k.Mm * k.HCm), p.og1 = T(k.Mm * k.HCm), p.lse1 = F(k.S * k.Hm * k.R), p.m1 = T(k.Mm * k.Cm);
  p.xm2 = T(k.Mm * k.Cm), p.qkvg2 = T(k.Mm * k.QKc), p.oatt2 = T(k.Mm * k.HCm), p.og2 = T(k.Mm * k.HCm);
  p.lse2 = F(k.R * k.Hm * k.S), p.m2 = T(k.Mm * k.Cm);
  p.gq = F(k.R * k.HCm), p.gob = F(k.R * k.HCm), p.gst = F(k.R * k.Hm * 2);
  p.xm3 = T(k.Mm * k.Cm), p.h3 = T(k.Mm * k.n * k.Cm), p.m3 = T(k.Mm * k.Cm);
  const int64_t Mz_opm = pair_only ? 0 : k.Mz;  // the outer product mean's pair buffers
  p.xm4 = T(k.Mm * k.Cm), p.ab4 = T(2 * k.Mm * k.co), p.O4 = T(Mz_opm * k.co * k.co), p.inv4 = F(Mz_opm);
  p.z1 = T(Mz_opm * k.Cz);
  for (int t = 0; t < 2; ++t) {
    TriBufs &b = p.tri[t];
    b.xz = T(k.Mz * k.Cz), b.abg = T(k.Mz * k.ABG), b.A = T(k.cmul * k.R * k.Rp), b.B = T(k.cmul * k.R * k.Rp);
    b.X = T(k.cmul * k.R * k.Rp), b.xo = T(k.Mz * k.cmul), b.y = T(k.Mz * k.Cz), b.zout = T(k.Mz * k.Cz);
  }
  for (int t = 0; t < 2; ++t) {
    AttBufs &b = p.att[t];
    b.xz = T(k.Mz * k.Cz), b.bias = F(k.Ht * k.Mz), b.qkvg = T(k.Mz * 4 * k.HCt), b.oatt = T(k.Mz * k.HCt);
    b.og = T(k.Mz * k.HCt), b.lse = F(k.R * k.Ht * k.R), b.zout = T(k.Mz * k.Cz);
  }
  p.xz9 = T(k.Mz * k.Cz), p.h9 = T(k.Mz * k.n * k.Cz), p.z6 = T(k.Mz * k.Cz);
  p.drop_u = T(std::max(k.Mm * k.Cm, k.Mz * k.Cz));
  if (mode == EVO_MODE_BWD) {
    p.dm_acc = F(k.Mm * k.Cm), p.dmT = T(k.Mm * k.Cm), p.dz_acc = F(k.Mz * k.Cz), p.dzT = T(k.Mz * k.Cz);
    int64_t g1 = std::max<int64_t>({k.Mm * k.n * k.Cm, k.Mz * k.n * k.Cz, k.Mm * k.QKm, k.Mm * k.QKc, k.Mz * 4 * k.HCt,
                           k.Mz * k.ABG});
    int64_t g2 = std::max<int64_t>({k.Mm * k.Cm, k.Mz * k.Cz, k.Mm * k.HCm, k.Mz * k.HCt, k.Mm * 2 * k.co});
    int64_t g3 = std::max<int64_t>({k.Mm * k.HCm, k.Mz * k.HCt, k.Mz * k.cmul, k.Mz * k.Cz});
    p.G1 = T(g1), p.G2 = T(g2), p.G3 = T(g3);
    p.dO4 = T(Mz_opm * k.co * k.co);
    p.dA = T(k.cmul * k.R * k.Rp), p.dB = T(k.cmul * k.R * k.Rp), p.dX = T(k.cmul * k.R * k.Rp);
    p.dq_acc = F(std::max(k.Mm * k.HCm, k.Mz * k.HCt));
    p.dbias = F(std::max(k.Hm, k.Ht) * k.Mz);
    p.Dsum = F(std::max(k.S * k.Hm * k.R, k.R * k.Ht * k.R));
    p.dab4 = T(k.Mm * 2 * k.co);
    int64_t wmax = std::max<int64_t>({k.QKm * k.Cm, k.QKc * k.Cm, k.n * k.Cm * k.Cm, k.n * k.Cz * k.Cz, k.ABG * k.Cz,
                             4 * k.HCt * k.Cz, k.Cz * k.co * k.co, k.Cm * k.HCm, 2 * k.co * k.Cm,
                             k.Cz * k.cmul, k.Cz * k.HCt});
    p.split = F(MAXSPLIT * wmax);
    p.wmax = wmax;
  }
  p.total = off;
  return off;
}

inline GemmOp mk(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, int amn, const void *B, int64_t ldb,
                 int bmn, void *C, int64_t ldc) {
  GemmOp g{};
  g.M = (int)M, g.N = (int)N, g.K = (int)K, g.batch = 1;
  g.A = A, g.lda = lda, g.a_mn = amn;
  g.B = B, g.ldb = ldb, g.b_mn = bmn;
  g.splits = 1;
  g.e.C = C;
  g.e.map = rowmajor_map(ldc);
  g.e.alpha = 1.f;
  g.e.act = ACT_NONE;
  return g;
}

struct Drv {
  const evo_dims &d;
  Dims2 k;
  int bf;
  size_t ts;
  cudaStream_t s;
  const float *p32;
  const bf16 *p16;
  std::map<std::string, int64_t> off;
  char *ws;
  Plan pl;
  float *dparams = nullptr;
  const evo_dropout *drop = nullptr;  // training-mode dropout scales (null: evaluation mode)
  // the transitions' hidden layers are written out only for the backward
  // (its recompute keeps them for dW2 and the ReLU mask)
  bool keep_hidden = false;
  cudaError_t err = cudaSuccess;

  Drv(const evo_dims &d_, const float *p32_, const bf16 *p16_, void *ws_, int mode, cudaStream_t s_,
      bool pair_only = false)
      : d(d_), k(d_, pair_only), bf(d_.act_dtype == EVO_BF16), ts(bf ? 2 : 4), s(s_), p32(p32_), p16(p16_),
        ws((char *)ws_), keep_hidden(mode == EVO_MODE_BWD) {
    std::vector<PEntry> t;
    build_param_table(d, t, pair_only);
    for (auto &e : t) off[e.name] = e.offset;
    make_plan(d, mode, pl, pair_only);
  }
  void ck(cudaError_t e) {
    if (err == cudaSuccess && e != cudaSuccess) err = e;
  }
  // dropout scale of a site (null when the block runs in evaluation mode or
  // the site is not dropped)
  const float *dsc(int site) const {
    if (!drop) return nullptr;
    switch (site) {
      case 0: return drop->msa_row;
      case 1: return drop->tri_out;
      case 2: return drop->tri_in;
      case 3: return drop->att_start;
      default: return drop->att_end;
    }
  }
  void *B(size_t o) { return ws + o; }
  float *Bf(size_t o) { return (float *)(ws + o); }
  void *at(const void *base, int64_t elems) { return (char *)base + elems * (int64_t)ts; }
  const float *P(const std::string &n) { return p32 + off.at(n); }
  const void *W(const std::string &n) {
    return bf ? (const void *)(p16 + off.at(n)) : (const void *)(p32 + off.at(n));
  }
  float *D(const std::string &n) { return dparams + off.at(n); }

  void gemm(GemmOp g) {
    g.e.M = g.M;
    g.e.N = g.N;
    if (bf && splitk_wanted(g)) {
      // too few output tiles to fill the GPU and a long K: fp32 partial sums
      // per K range, then one reduction writes the bf16 output through the map
      const int64_t tiles = ((g.M + 127) / 128) * ((g.N + 255) / 256);
      int64_t sp = std::min<int64_t>((152 + tiles - 1) / tiles, g.K / 1024);
      sp = std::min<int64_t>(sp, (int64_t)MAXSPLIT * pl.wmax / ((int64_t)g.M * g.N));
      if (sp >= 2) {
        const OutMap map = g.e.map;
        void *out = g.e.C;
        g.splits = (int)sp;
        g.e.partial = Bf(pl.split);
        g.e.C = nullptr;
        ck(gemm_tc_bf16(g, s));
        ck(reduce_splits_map(Bf(pl.split), (int)sp, g.M, g.N, map, out, s));
        return;
      }
    }
    ck(bf ? gemm_tc_bf16(g, s) : gemm_simt_f32(g, s));
  }
  // A plain product (no epilogue but the output map) whose tiles cannot fill the GPU.
  static bool splitk_wanted(const GemmOp &g) {
    const Epi &e = g.e;
    const int64_t tiles = ((g.M + 127) / 128) * ((g.N + 255) / 256) * g.batch;
    return g.batch == 1 && g.splits == 1 && !e.partial && tiles * 2 <= 152 && g.K >= 2048 && g.N % 2 == 0 &&
           e.alpha == 1.f && !e.bias && !e.row_scale && !e.relu_ref && e.act == ACT_NONE && !e.aux && !e.gate &&
           !e.residual && !e.c_f32 && !e.accumulate;
  }
  void ln(const void *x, const std::string &pre, void *y, int64_t M, int C) {
    ck(ln_fwd(x, P(pre + ".gamma"), P(pre + ".beta"), y, M, C, bf, s));
  }

  // ---------------- backward helpers (parameter gradients accumulate into dparams)
  void dW(const void *dY, int64_t ldY, int64_t Nout, const void *X, int64_t ldX, int64_t Kin, int64_t rows,
          const std::string &w) {
    GemmOp g = mk(Nout, Kin, rows, dY, ldY, 1, X, ldX, 1, nullptr, 0);
    int64_t sp;
    if (bf) {
      // split K until the CTAs fill the SMs once (the tcgen05 GEMM is persistent,
      // BN = 256 or 128), keeping at least eight 64-deep k-tiles per split; the
      // partial products meet in the fp32 gradient through atomics
      const int64_t bn = Kin > 128 && Kin % 256 == 0 ? 256 : 128;
      const int64_t tiles = ((Nout + 127) / 128) * ((Kin + bn - 1) / bn);
      sp = std::min<int64_t>((152 + tiles - 1) / tiles, std::max<int64_t>(1, rows / 512));
    } else {
      const int64_t tiles = ((Nout + 63) / 64) * ((Kin + 63) / 64);
      sp = std::min<int64_t>((2 * 152 + tiles - 1) / tiles, std::max<int64_t>(1, rows / 256));
      sp = std::min<int64_t>(sp, MAXSPLIT);
    }
    sp = std::max<int64_t>(1, sp);
    g.splits = (int)sp;
    if (bf) {
      // each K range adds its partial product straight into the fp32 gradient
      g.e.C = D(w), g.e.c_f32 = 1, g.e.atomic = 1, g.e.map = rowmajor_map(Kin);
      gemm(g);
    } else {
      g.e.partial = Bf(pl.split);
      gemm(g);
      ck(reduce_splits(Bf(pl.split), (int)sp, Nout * Kin, D(w), s));
    }
  }
  void db(const void *dY, int64_t ldY, int64_t rows, int64_t N, const std::string &b) {
    ck(colsum(dY, ldY, rows, (int)N, bf, s, D(b)));
  }
  // next_db: the bias gradient of the layer that consumes this gradient next
  // (the column sums of the updated accumulator, fused into the kernel)
  void lnb(const void *dy, const void *x, const std::string &pre, float *dacc, void *dcopy, void *dx_out, int64_t M,
           int C, const void *dinit = nullptr, float *next_db = nullptr) {
    ck(ln_bwd(dy, x, P(pre + ".gamma"), dacc, dcopy, dx_out, M, C, bf, s, D(pre + ".gamma"), D(pre + ".beta"), dinit,
              next_db));
  }

  // ---------------- attention argument sets
  // kind 0: MSA row (batch s, query i, key j), 1: MSA column (batch i, query s, key t),
  //      2: triangle start (batch i, query j, key k), 3: triangle end (batch j, query i, key k)
  AttnArgs attn_args(int kind, void *qkvg, void *oatt, void *og, float *lse, float *bias, const float *mask) {
    AttnArgs a{};
    const bool msa = kind < 2;
    const int64_t H = msa ? k.Hm : k.Ht, c = msa ? k.cm : k.ct, HC = H * c, QK = 4 * HC;
    const int64_t R = k.R, S = k.S;
    a.q = qkvg, a.k = at(qkvg, HC), a.v = at(qkvg, 2 * HC), a.g = at(qkvg, 3 * HC);
    a.H = (int)H, a.c = (int)c;
    a.o_att = oatt, a.o_gate = og, a.lse2 = lse;
    a.scale = 1.f / std::sqrt((float)c);
    a.bias = bias;
    a.bias_bf16 = bf;  // the pair bias is an activation: bf16 on the BF16 path
    a.sBh = k.Mz, a.sBx = R;
    a.mask = mask;
    switch (kind) {
      case 0:
        a.B1 = (int)S, a.X = (int)R, a.Y = (int)R;
        a.sQb = R * QK, a.sQx = QK, a.sKb = R * QK, a.sKy = QK;
        a.sMb = R, a.sMy = 1;
        a.sOb = R * HC, a.sOx = HC;
        break;
      case 1:
        a.B1 = (int)R, a.X = (int)S, a.Y = (int)S;
        a.sQb = QK, a.sQx = R * QK, a.sKb = QK, a.sKy = R * QK;
        a.sMb = 1, a.sMy = R;
        a.sOb = HC, a.sOx = R * HC;
        break;
      case 2:
        a.B1 = (int)R, a.X = (int)R, a.Y = (int)R;
        a.sQb = R * QK, a.sQx = QK, a.sKb = R * QK, a.sKy = QK;
        a.sMb = R, a.sMy = 1;
        a.sOb = R * HC, a.sOx = HC;
        break;
      default:
        a.B1 = (int)R, a.X = (int)R, a.Y = (int)R;
        a.sQb = QK, a.sQx = R * QK, a.sKb = QK, a.sKy = R * QK;
        a.sMb = 1, a.sMy = R;
        a.sOb = HC, a.sOx = R * HC;
        break;
    }
    return a;
  }

  GlobalAttnArgs global_args() {
    GlobalAttnArgs a{};
    a.qkvg = B(pl.qkvg2), a.ld = k.QKc, a.S = (int)k.S, a.R = (int)k.R, a.H = (int)k.Hm, a.c = (int)k.cm;
    a.mask = msa_mask_, a.o_att_bar = Bf(pl.gob), a.qbar = Bf(pl.gq), a.lse2 = Bf(pl.gst), a.o_gate = B(pl.og2);
    a.scale = 1.f / std::sqrt((float)k.cm);
    return a;
  }

  // ================================================================ forward
  const float *msa_mask_ = nullptr;

  void forward(const void *m0, const void *z0, void *m_out, void *z_out, const float *mm, const float *pm) {
    msa_mask_ = mm;
    const int64_t S = k.S, R = k.R, Cm = k.Cm, Cz = k.Cz, Mm = k.Mm, Mz = k.Mz, HCm = k.HCm, HCt = k.HCt;
    // 1. MSA row attention with pair bias (AF2 Alg. 7)
    ln(m0, "row.ln_m", B(pl.xm1), Mm, (int)Cm);
    if (pl.sl.on) {
      // the pair bias of the row attention, one i-slab of LayerNorm(z) at a time
      slabs([&](int64_t i0, int64_t ri) {
        ln(at(z0, i0 * R * Cz), "row.ln_z", B(pl.sl.xz1), ri * R, (int)Cz);
        ck(head_proj_fwd_rows(B(pl.sl.xz1), P("row.w_b"), at(B(pl.bias1), i0 * R), ri * R, Mz, (int)Cz, (int)k.Hm,
                              s));
      });
    } else {
      ln(z0, "row.ln_z", B(pl.xz1), Mz, (int)Cz);
      ck(head_proj_fwd(B(pl.xz1), P("row.w_b"), Bf(pl.bias1), (int)R, (int)Cz, (int)k.Hm, 0, bf, s));
    }
    {
      GemmOp g = mk(Mm, k.QKm, Cm, B(pl.xm1), Cm, 0, W("row.w_qkvg"), Cm, 0, B(pl.qkvg1), k.QKm);
      g.e.bias = P("row.b_g"), g.e.bias_n0 = (int)(3 * HCm), g.e.act = ACT_SIGMOID, g.e.act_n0 = (int)(3 * HCm);
      gemm(g);
      AttnArgs a = attn_args(0, B(pl.qkvg1), B(pl.oatt1), B(pl.og1), Bf(pl.lse1), Bf(pl.bias1), mm);
      ck(attn_fwd(a, bf, s));
      const float *sc = dsc(0);
      GemmOp o = mk(Mm, Cm, HCm, B(pl.og1), HCm, 0, W("row.w_o"), HCm, 0, B(sc ? pl.drop_u : pl.m1), Cm);
      o.e.bias = P("row.b_o"), o.e.residual = sc ? nullptr : m0;
      gemm(o);
      if (sc) ck(dropout_apply(B(pl.drop_u), sc, m0, B(pl.m1), Mm, (int)Cm, (int)R, 0, bf, s));
    }
    // 2. MSA column attention (AF2 Alg. 8), or global column attention (AF2 Alg. 19)
    ln(B(pl.m1), "col.ln", B(pl.xm2), Mm, (int)Cm);
    {
      const int64_t g0 = d.msa_col_mode == EVO_COL_GLOBAL ? HCm + 2 * k.cm : 3 * HCm;
      GemmOp g = mk(Mm, k.QKc, Cm, B(pl.xm2), Cm, 0, W("col.w_qkvg"), Cm, 0, B(pl.qkvg2), k.QKc);
      g.e.bias = P("col.b_g"), g.e.bias_n0 = (int)g0, g.e.act = ACT_SIGMOID, g.e.act_n0 = (int)g0;
      gemm(g);
      if (d.msa_col_mode == EVO_COL_GLOBAL) {
        ck(global_attn_fwd(global_args(), bf, s));
      } else {
        AttnArgs a = attn_args(1, B(pl.qkvg2), B(pl.oatt2), B(pl.og2), Bf(pl.lse2), nullptr, mm);
        ck(attn_fwd(a, bf, s));
      }
      GemmOp o = mk(Mm, Cm, HCm, B(pl.og2), HCm, 0, W("col.w_o"), HCm, 0, B(pl.m2), Cm);
      o.e.bias = P("col.b_o"), o.e.residual = B(pl.m1);
      gemm(o);
    }
    // 3. MSA transition (AF2 Alg. 9)
    void *m3 = m_out ? m_out : B(pl.m3);
    transition_fwd("msa_trans", B(pl.m2), B(pl.xm3), B(pl.h3), m3, Mm, Cm);
    // 4. outer product mean (AF2 Alg. 10)
    ln(m3, "opm.ln", B(pl.xm4), Mm, (int)Cm);
    {
      const int64_t co = k.co;
      GemmOp g = mk(Mm, 2 * co, Cm, B(pl.xm4), Cm, 0, W("opm.w_ab"), Cm, 0, B(pl.ab4), 0);
      g.e.map = OutMap{1ll << 40, 0, co, co, Mm * co, 1};  // a -> [s][i][c], b -> [s][j][d]
      g.e.bias = P("opm.b_ab"), g.e.row_scale = mm;
      gemm(g);
      ck(opm_inv_norm(mm, Bf(pl.inv4), (int)S, (int)R, 1e-3f, s));
      // the outer products and their projection, for all rows i at once or
      // one i-slab at a time (the slab's a rows against every b row)
      auto outer = [&](int64_t i0, int64_t ri, size_t O4) {
        GemmOp o = mk(ri * co, R * co, S, at(B(pl.ab4), i0 * co), R * co, 1, at(B(pl.ab4), Mm * co), R * co, 1,
                      B(O4), 0);
        o.e.map = OutMap{co, R * co * co, co, co, co * co, 1};  // O[i][j][c*co + d]
        o.cls = "opm_outer";
        gemm(o);
        GemmOp p = mk(ri * R, Cz, co * co, B(O4), co * co, 0, W("opm.w_o"), co * co, 0, at(B(pl.z1), i0 * R * Cz), Cz);
        p.e.bias = P("opm.b_o"), p.e.row_scale = Bf(pl.inv4) + i0 * R, p.e.residual = at(z0, i0 * R * Cz);
        gemm(p);
      };
      if (pl.sl.on) slabs([&](int64_t i0, int64_t ri) { outer(i0, ri, pl.sl.O4); });
      else outer(0, R, pl.O4);
    }
    if (pl.sl.on) pair_forward_slabbed(z_out, pm);
    else pair_forward(B(pl.z1), z_out, pm);
    (void)HCt;
  }

  // Steps 5-9 of the block from the pair input zin; also the whole template
  // pair stack block (AF2 Alg. 16).
  void pair_forward(const void *zin, void *z_out, const float *pm) {
    // 5, 6. triangle multiplication outgoing / incoming (AF2 Alg. 11, 12)
    trimul_fwd(0, zin, pm);
    trimul_fwd(1, B(pl.tri[0].zout), pm);
    // 7, 8. triangle attention starting / ending node (AF2 Alg. 13, 14)
    triatt_fwd(0, B(pl.tri[1].zout), pm);
    triatt_fwd(1, B(pl.att[0].zout), pm);
    // 9. pair transition (AF2 Alg. 15)
    void *z6 = z_out ? z_out : B(pl.z6);
    transition_fwd("pair_trans", B(pl.att[1].zout), B(pl.xz9), B(pl.h9), z6, k.Mz, k.Cz);
  }

  // ---------------- i-slab subbatching of steps 5-9 (Sec. 3.4.4), inference plan
  // Every pair step works on Ri rows of the pair grid at a time.  Outgoing
  // multiplication, starting attention and the transition need, for a row i,
  // only what is computed from row i plus a full-size operand built in a
  // first pass over the slabs (the b side of the triangle product, the pair
  // bias of the attention).  Incoming multiplication and ending attention are
  // the outgoing / starting forms on the transposed grid: with z'[i][j] =
  // z[j][i] and the a and b projections swapped, the outgoing product on z'
  // at (i, j) is the incoming one on z at (j, i), and the starting attention
  // on z' (mask and bias transposed with it) is the ending attention on z;
  // their outputs go back through a transposed output map.
  template <class Fn>
  void slabs(Fn f) {
    for (int64_t i0 = 0; i0 < k.R; i0 += pl.sl.Ri) f(i0, std::min(pl.sl.Ri, k.R - i0));
  }
  // The output projection of a slab: written in place through the row-major
  // map, or (transposed grid) into a slab-sized buffer and then put back into
  // the columns i0 .. i0 + ri of z, so that both take the same epilogue.  The
  // residual is the source grid's own rows either way (z'[i][j] = z[j][i]).
  void slab_project(GemmOp o, const void *src, void *out, void *tmp, bool transposed, int64_t i0, int64_t ri) {
    const int64_t R = k.R, Cz = k.Cz;
    o.e.residual = at(src, i0 * R * Cz);
    o.e.C = transposed ? tmp : at(out, i0 * R * Cz);
    gemm(o);
    if (transposed) ck(transpose_rows(tmp, at(out, i0 * Cz), ri, R, (int)(Cz * ts / 4), R, s));
  }

  void pair_forward_slabbed(void *z_out, const float *pm) {
    const Plan::Slab &sl = pl.sl;
    const int64_t R = k.R;
    const int W = (int)(k.Cz * ts / 4);
    void *za = B(pl.z1), *zb = B(pl.tri[0].zout);
    // 5. outgoing: z1 -> zb
    trimul_fwd_slabbed(0, za, pm, zb, false);
    // 6. incoming, on the transposed grid: zb -> z1
    ck(transpose_rows(zb, B(sl.zT), R, R, W, R, s));
    ck(transpose_rows(pm, Bf(sl.pmT), R, R, 1, R, s));
    trimul_fwd_slabbed(1, B(sl.zT), Bf(sl.pmT), za, true);
    // 7. starting node: z1 -> zb
    triatt_fwd_slabbed(0, za, pm, zb, false);
    // 8. ending node, as starting on the transposed grid: zb -> z1
    ck(transpose_rows(zb, B(sl.zT), R, R, W, R, s));
    triatt_fwd_slabbed(1, B(sl.zT), Bf(sl.pmT), za, true);
    // 9. pair transition: z1 -> z_out (or zb)
    void *z6 = z_out ? z_out : B(pl.z6);
    slabs([&](int64_t i0, int64_t ri) {
      const int64_t o = i0 * R * k.Cz;
      transition_fwd("pair_trans", at(za, o), B(sl.txz), B(sl.h), at(z6, o), ri * R, k.Cz);
    });
  }

  // src: the grid the step reads row by row (z, or its transpose) with its
  // mask msk; out: the step's output, addressed as z.
  void trimul_fwd_slabbed(int t, const void *src, const float *msk, void *out, bool transposed) {
    const std::string pre = t == 0 ? "tri_out" : "tri_in";
    const Plan::Slab &sl = pl.sl;
    const int64_t R = k.R, Rp = k.Rp, Cz = k.Cz, cmul = k.cmul, ABG = k.ABG;
    const int swap = transposed ? 1 : 0;
    // First pass: the b side of every row into the full-size channel-major
    // Bfull, from the b half of w_abg alone (columns [2 cmul, 4 cmul); the a
    // half [0, 2 cmul) when swapped).  The gate kernel also writes an a from
    // the stale other half of abg into the slab's A: discarded.
    const int64_t cb = swap ? 0 : 2 * cmul;
    slabs([&](int64_t i0, int64_t ri) {
      ln(at(src, i0 * R * Cz), pre + ".ln_in", B(sl.xz), ri * R, (int)Cz);
      GemmOp g = mk(ri * R, 2 * cmul, Cz, B(sl.xz), Cz, 0, at(W(pre + ".w_abg"), cb * Cz), Cz, 0,
                    at(B(sl.abg), cb), ABG);
      g.e.bias = P(pre + ".b_abg") + cb;
      gemm(g);
      ck(trimul_gate_fwd_rows(B(sl.abg), ABG, msk + i0 * R, B(sl.A), ri * Rp, at(B(sl.Bfull), i0 * Rp), R * Rp, Rp,
                              (int)ri, (int)R, (int)cmul, swap, s));
    });
    // Second pass: a of the slab (its b goes to the X buffer, overwritten
    // next), the product against every row of b, LayerNorm, projection.
    slabs([&](int64_t i0, int64_t ri) {
      ln(at(src, i0 * R * Cz), pre + ".ln_in", B(sl.xz), ri * R, (int)Cz);
      GemmOp g = mk(ri * R, ABG, Cz, B(sl.xz), Cz, 0, W(pre + ".w_abg"), Cz, 0, B(sl.abg), ABG);
      g.e.bias = P(pre + ".b_abg");
      g.e.act = ACT_SIGMOID, g.e.act_n0 = (int)(4 * cmul);  // the output gate g
      gemm(g);
      ck(trimul_gate_fwd_rows(B(sl.abg), ABG, msk + i0 * R, B(sl.A), ri * Rp, B(sl.X), ri * Rp, Rp, (int)ri, (int)R,
                              (int)cmul, swap, s));
      GemmOp x = mk(ri, R, R, B(sl.A), Rp, 0, B(sl.Bfull), Rp, 0, B(sl.X), Rp);
      x.batch = (int)cmul, x.a_bs = ri * Rp, x.b_bs = R * Rp, x.e.c_bstride = ri * Rp;
      x.cls = "tri_einsum";
      gemm(x);
      ck(ln_fwd_cm_rows(B(sl.X), Rp, ri * Rp, P(pre + ".ln_out.gamma"), P(pre + ".ln_out.beta"), B(sl.xo), (int)ri,
                        (int)R, (int)cmul, s));
      GemmOp o = mk(ri * R, Cz, cmul, B(sl.xo), cmul, 0, W(pre + ".w_o"), cmul, 0, nullptr, Cz);
      o.e.bias = P(pre + ".b_o");
      o.e.gate = at(B(sl.abg), 4 * cmul), o.e.gate_ld = ABG;
      slab_project(o, src, out, B(sl.y), transposed, i0, ri);
    });
  }

  void triatt_fwd_slabbed(int t, const void *src, const float *msk, void *out, bool transposed) {
    const std::string pre = t == 0 ? "att_start" : "att_end";
    const Plan::Slab &sl = pl.sl;
    const int64_t R = k.R, Cz = k.Cz, Mz = k.Mz, HCt = k.HCt;
    // first pass: the pair bias b[h][j][k] of every row (starting form on src)
    slabs([&](int64_t i0, int64_t ri) {
      ln(at(src, i0 * R * Cz), pre + ".ln", B(sl.axz), ri * R, (int)Cz);
      ck(head_proj_fwd_rows(B(sl.axz), P(pre + ".w_b"), at(B(sl.tbias), i0 * R), ri * R, Mz, (int)Cz, (int)k.Ht, s));
    });
    slabs([&](int64_t i0, int64_t ri) {
      ln(at(src, i0 * R * Cz), pre + ".ln", B(sl.axz), ri * R, (int)Cz);
      GemmOp g = mk(ri * R, 4 * HCt, Cz, B(sl.axz), Cz, 0, W(pre + ".w_qkvg"), Cz, 0, B(sl.qkvg), 4 * HCt);
      g.e.bias = P(pre + ".b_g"), g.e.bias_n0 = (int)(3 * HCt), g.e.act = ACT_SIGMOID, g.e.act_n0 = (int)(3 * HCt);
      gemm(g);
      AttnArgs a = attn_args(2, B(sl.qkvg), B(sl.oatt), B(sl.og), Bf(sl.lse), Bf(sl.tbias), msk + i0 * R);
      a.B1 = (int)ri;
      ck(attn_fwd(a, bf, s));
      GemmOp o = mk(ri * R, Cz, HCt, B(sl.og), HCt, 0, W(pre + ".w_o"), HCt, 0, nullptr, Cz);
      o.e.bias = P(pre + ".b_o");
      slab_project(o, src, out, B(sl.axz), transposed, i0, ri);  // the LayerNorm output is dead here
    });
  }

  void transition_fwd(const std::string &pre, const void *x, void *xn, void *h, void *out, int64_t M, int64_t C) {
    ln(x, pre + ".ln", xn, M, (int)C);
    const int64_t nC = k.n * C;
    // Without the backward the hidden layer is needed by no one: both
    // products run in one kernel with the hidden layer kept on the SM.  The
    // backward's recompute keeps h (dW2, the ReLU mask), and there the two
    // GEMMs, which write h as their intermediate anyway, are faster.
    if (bf && !keep_hidden &&
        mlp_fused_supported(M, (int)C, (int)nC, xn, W(pre + ".w1"), P(pre + ".b1"), W(pre + ".w2"), P(pre + ".b2"), x,
                            out)) {
      ck(mlp_fused_tc(xn, W(pre + ".w1"), P(pre + ".b1"), W(pre + ".w2"), P(pre + ".b2"), x, out, M, (int)C, (int)nC,
                      s));
      return;
    }
    GemmOp g = mk(M, nC, C, xn, C, 0, W(pre + ".w1"), C, 0, h, nC);
    g.e.bias = P(pre + ".b1"), g.e.act = ACT_RELU;
    gemm(g);
    GemmOp o = mk(M, C, nC, h, nC, 0, W(pre + ".w2"), nC, 0, out, C);
    o.e.bias = P(pre + ".b2"), o.e.residual = x;
    gemm(o);
  }

  void trimul_fwd(int t, const void *zin, const float *pm) {
    const std::string pre = t == 0 ? "tri_out" : "tri_in";
    const TriBufs &b = pl.tri[t];
    const int64_t R = k.R, Rp = k.Rp, Cz = k.Cz, Mz = k.Mz, cmul = k.cmul, ABG = k.ABG;
    ln(zin, pre + ".ln_in", B(b.xz), Mz, (int)Cz);
    GemmOp g = mk(Mz, ABG, Cz, B(b.xz), Cz, 0, W(pre + ".w_abg"), Cz, 0, B(b.abg), ABG);
    g.e.bias = P(pre + ".b_abg");
    g.e.act = ACT_SIGMOID, g.e.act_n0 = (int)(4 * cmul);  // the output gate g
    gemm(g);
    ck(trimul_gate_fwd(B(b.abg), ABG, pm, B(b.A), B(b.B), Rp, (int)R, (int)cmul, t, bf, s));
    // X_c = A_c B_c^T per channel c (incoming stores A, B transposed, so the product is the same)
    GemmOp x = mk(R, R, R, B(b.A), Rp, 0, B(b.B), Rp, 0, B(b.X), Rp);
    x.batch = (int)cmul, x.a_bs = R * Rp, x.b_bs = R * Rp, x.e.c_bstride = R * Rp;
    x.cls = "tri_einsum";
    gemm(x);
    ck(ln_fwd_cm(B(b.X), Rp, P(pre + ".ln_out.gamma"), P(pre + ".ln_out.beta"), B(b.xo), (int)R, (int)cmul, bf, s));
    const float *sc = dsc(1 + t);
    GemmOp o = mk(Mz, Cz, cmul, B(b.xo), cmul, 0, W(pre + ".w_o"), cmul, 0, B(sc ? pl.drop_u : b.zout), Cz);
    o.e.bias = P(pre + ".b_o"), o.e.aux = B(b.y), o.e.aux_ld = Cz;
    o.e.gate = at(B(b.abg), 4 * cmul), o.e.gate_ld = ABG, o.e.residual = sc ? nullptr : zin;
    gemm(o);
    if (sc) ck(dropout_apply(B(pl.drop_u), sc, zin, B(b.zout), Mz, (int)Cz, (int)R, 0, bf, s));
  }

  void triatt_fwd(int t, const void *zin, const float *pm) {
    const std::string pre = t == 0 ? "att_start" : "att_end";
    const AttBufs &b = pl.att[t];
    const int64_t R = k.R, Cz = k.Cz, Mz = k.Mz, HCt = k.HCt;
    ln(zin, pre + ".ln", B(b.xz), Mz, (int)Cz);
    ck(head_proj_fwd(B(b.xz), P(pre + ".w_b"), Bf(b.bias), (int)R, (int)Cz, (int)k.Ht, t, bf, s));
    GemmOp g = mk(Mz, 4 * HCt, Cz, B(b.xz), Cz, 0, W(pre + ".w_qkvg"), Cz, 0, B(b.qkvg), 4 * HCt);
    g.e.bias = P(pre + ".b_g"), g.e.bias_n0 = (int)(3 * HCt), g.e.act = ACT_SIGMOID, g.e.act_n0 = (int)(3 * HCt);
    gemm(g);
    AttnArgs a = attn_args(2 + t, B(b.qkvg), B(b.oatt), B(b.og), Bf(b.lse), Bf(b.bias), pm);
    ck(attn_fwd(a, bf, s));
    const float *sc = dsc(3 + t);
    GemmOp o = mk(Mz, Cz, HCt, B(b.og), HCt, 0, W(pre + ".w_o"), HCt, 0, B(sc ? pl.drop_u : b.zout), Cz);
    o.e.bias = P(pre + ".b_o"), o.e.residual = sc ? nullptr : zin;
    gemm(o);
    if (sc) ck(dropout_apply(B(pl.drop_u), sc, zin, B(b.zout), Mz, (int)Cz, (int)R, t, bf, s));
  }

  // ================================================================ backward
  // dacc/dT: FP32 running gradient of the residual stream and its storage-type copy.
  // dT: the incoming gradient (activation type); dcopy receives the updated
  // running gradient (dT itself unless the incoming one must stay intact);
  // dinit: start the fp32 accumulator from this tensor instead of its contents.
  // b2_done: the b2 gradient (column sums of dT) was added by the kernel that
  // wrote dT; next_db as in lnb.
  void transition_bwd(const std::string &pre, const void *x, const void *xn, const void *h, float *dacc,
                      const void *dT, void *dcopy, int64_t M, int64_t C, const void *dinit = nullptr,
                      bool b2_done = false, float *next_db = nullptr) {
    const int64_t nC = k.n * C;
    dW(dT, C, C, h, nC, nC, M, pre + ".w2");
    if (!b2_done) db(dT, C, M, C, pre + ".b2");
    GemmOp g = mk(M, nC, C, dT, C, 0, W(pre + ".w2"), nC, 1, B(pl.G1), nC);
    g.e.relu_ref = h, g.e.relu_ld = nC;
    gemm(g);
    dW(B(pl.G1), nC, nC, xn, C, C, M, pre + ".w1");
    db(B(pl.G1), nC, M, nC, pre + ".b1");
    GemmOp o = mk(M, C, nC, B(pl.G1), nC, 0, W(pre + ".w1"), C, 1, B(pl.G2), C);
    gemm(o);
    lnb(B(pl.G2), x, pre + ".ln", dacc, dcopy, nullptr, M, (int)C, dinit, next_db);
  }

  // Gated attention backward down to d(LN input) in G2 (not yet through LayerNorm).
  // Leaves dqkvg in G1 and the pair-bias gradient in dbias (when bias != null).
  // bo_done: the b_o gradient (column sums of dT) was added by the kernel
  // that wrote dT.
  void attention_bwd(int kind, const std::string &pre, const void *xn, void *qkvg, void *oatt, void *og, float *lse,
                     float *bias, const float *mask, const void *dT, int64_t M, int64_t Cin, bool bo_done = false) {
    const bool msa = kind < 2;
    const int64_t HC = msa ? k.HCm : k.HCt, QK = 4 * HC;
    dW(dT, Cin, Cin, og, HC, HC, M, pre + ".w_o");
    if (!bo_done) db(dT, Cin, M, Cin, pre + ".b_o");
    GemmOp g = mk(M, HC, Cin, dT, Cin, 0, W(pre + ".w_o"), HC, 1, B(pl.G2), HC);
    gemm(g);
    AttnArgs a = attn_args(kind, qkvg, oatt, og, lse, bias, mask);
    a.do_att = B(pl.G3);
    a.Dsum = Bf(pl.Dsum);
    a.dq_acc = Bf(pl.dq_acc);
    a.dk = at(B(pl.G1), HC);
    a.dv = at(B(pl.G1), 2 * HC);
    a.dbias = bias ? Bf(pl.dbias) : nullptr;
    a.dq = B(pl.G1);
    a.dog = B(pl.G2);                  // gradient of the gated output
    a.dgpre = at(B(pl.G1), 3 * HC);    // gate pre-activation gradient
    if (bias) ck(cudaMemsetAsync(Bf(pl.dbias), 0, (size_t)a.H * k.Mz * 4, s));
    ck(attn_bwd(a, bf, s));
    dW(B(pl.G1), QK, QK, xn, Cin, Cin, M, pre + ".w_qkvg");
    db(at(B(pl.G1), 3 * HC), QK, M, HC, pre + ".b_g");
    GemmOp x = mk(M, Cin, QK, B(pl.G1), QK, 0, W(pre + ".w_qkvg"), Cin, 1, B(pl.G2), Cin);
    gemm(x);
  }

  void pair_bias_bwd(const std::string &wname, const void *xn, int H, int transpose, int accumulate) {
    ck(head_proj_bwd(Bf(pl.dbias), xn, P(wname), B(pl.G2), accumulate, (int)k.R, (int)k.Cz, H, transpose, bf, s,
                     D(wname)));
  }

  // dT: the incoming gradient (activation type); dcopy receives the updated
  // running gradient (dT itself when null).
  void trimul_bwd(int t, const void *zin, const float *pm, float *dacc, void *dT, void *dcopy = nullptr) {
    const std::string pre = t == 0 ? "tri_out" : "tri_in";
    const TriBufs &b = pl.tri[t];
    const int64_t R = k.R, Rp = k.Rp, Cz = k.Cz, Mz = k.Mz, cmul = k.cmul, ABG = k.ABG;
    const float *sc = dsc(1 + t);
    if (sc) ck(dropout_apply(dT, sc, nullptr, B(pl.drop_u), Mz, (int)Cz, (int)R, 0, bf, s));
    ck(gate_out_bwd(sc ? B(pl.drop_u) : dT, at(B(b.abg), 4 * cmul), ABG, B(b.y), B(pl.G2), at(B(pl.G1), 4 * cmul), ABG,
                    Mz, (int)Cz, bf, s, D(pre + ".b_o")));
    dW(B(pl.G2), Cz, Cz, B(b.xo), cmul, cmul, Mz, pre + ".w_o");
    GemmOp g = mk(Mz, cmul, Cz, B(pl.G2), Cz, 0, W(pre + ".w_o"), cmul, 1, B(pl.G3), cmul);
    gemm(g);
    ck(ln_bwd_cm(B(pl.G3), B(b.X), Rp, P(pre + ".ln_out.gamma"), B(pl.dX), (int)R, (int)cmul, bf, s,
                 D(pre + ".ln_out.gamma"), D(pre + ".ln_out.beta")));
    // dA_c = dX_c B_c ; dB_c = dX_c^T A_c
    GemmOp ga = mk(R, R, R, B(pl.dX), Rp, 0, B(b.B), Rp, 1, B(pl.dA), Rp);
    ga.batch = (int)cmul, ga.a_bs = R * Rp, ga.b_bs = R * Rp, ga.e.c_bstride = R * Rp;
    ga.cls = "tri_einsum";
    gemm(ga);
    GemmOp gb = mk(R, R, R, B(pl.dX), Rp, 1, B(b.A), Rp, 1, B(pl.dB), Rp);
    gb.batch = (int)cmul, gb.a_bs = R * Rp, gb.b_bs = R * Rp, gb.e.c_bstride = R * Rp;
    gb.cls = "tri_einsum";
    gemm(gb);
    ck(trimul_gate_bwd(B(pl.dA), B(pl.dB), Rp, B(b.abg), ABG, pm, B(pl.G1), (int)R, (int)cmul, t, bf, s));
    dW(B(pl.G1), ABG, ABG, B(b.xz), Cz, Cz, Mz, pre + ".w_abg");
    db(B(pl.G1), ABG, Mz, ABG, pre + ".b_abg");
    GemmOp x = mk(Mz, Cz, ABG, B(pl.G1), ABG, 0, W(pre + ".w_abg"), Cz, 1, B(pl.G2), Cz);
    gemm(x);
    lnb(B(pl.G2), zin, pre + ".ln_in", dacc, dcopy ? dcopy : dT, nullptr, Mz, (int)Cz);
  }

  // Steps 9-5 of the backward (the template pair stack block whole): from the
  // incoming dz_out to the gradient at the pair input zin, accumulated in the
  // fp32 dz_acc and copied to dz_last (activation type) by the last LayerNorm
  // backward.
  void pair_backward(const void *zin, const float *pm, const void *dz_out, void *dz_last) {
    const int64_t R = k.R, Cz = k.Cz, Mz = k.Mz;
    float *dz = Bf(pl.dz_acc);
    void *dzT = B(pl.dzT);
    // 9. pair transition
    transition_bwd("pair_trans", B(pl.att[1].zout), B(pl.xz9), B(pl.h9), dz, dz_out, dzT, Mz, Cz, dz_out, false,
                   dsc(4) ? nullptr : D("att_end.b_o"));
    // 8, 7. triangle attention ending / starting node
    for (int t = 1; t >= 0; --t) {
      const AttBufs &b = pl.att[t];
      const std::string pre = t == 0 ? "att_start" : "att_end";
      const void *zt = t == 0 ? B(pl.tri[1].zout) : B(pl.att[0].zout);
      // with dropout the update's gradient is dz scaled by the site's draw
      const float *sc = dsc(3 + t);
      if (sc) ck(dropout_apply(dzT, sc, nullptr, B(pl.drop_u), Mz, (int)Cz, (int)R, t, bf, s));
      attention_bwd(2 + t, pre, B(b.xz), B(b.qkvg), B(b.oatt), B(b.og), Bf(b.lse), Bf(b.bias), pm,
                    sc ? B(pl.drop_u) : dzT, Mz, Cz, sc == nullptr);
      pair_bias_bwd(pre + ".w_b", B(b.xz), (int)k.Ht, t, 1);
      lnb(B(pl.G2), zt, pre + ".ln", dz, dzT, nullptr, Mz, (int)Cz, nullptr,
          t == 1 && !dsc(3) ? D("att_start.b_o") : nullptr);
    }
    // 6, 5. triangle multiplication incoming / outgoing
    trimul_bwd(1, B(pl.tri[0].zout), pm, dz, dzT);
    trimul_bwd(0, zin, pm, dz, dzT, dz_last);
  }

  void backward(const void *m0, const void *z0, const float *mm, const float *pm, const void *dm_out,
                const void *dz_out, void *dm_in, void *dz_in) {
    const int64_t S = k.S, R = k.R, Cm = k.Cm, Cz = k.Cz, Mm = k.Mm, Mz = k.Mz, co = k.co;
    // running gradients of the two residual streams: fp32 accumulators dm, dz
    // and their activation-type copies dmT, dzT.  The first LayerNorm backward
    // of each stream starts its accumulator from the incoming cotangent, and
    // the last one writes the outgoing gradient, so no conversion pass exists.
    float *dm = Bf(pl.dm_acc), *dz = Bf(pl.dz_acc);
    void *dmT = B(pl.dmT), *dzT = B(pl.dzT);

    pair_backward(B(pl.z1), pm, dz_out, dzT);
    // 4. outer product mean
    {
      ck(row_scale(dzT, Bf(pl.inv4), B(pl.G2), Mz, (int)Cz, bf, s, D("opm.b_o")));
      dW(B(pl.G2), Cz, Cz, B(pl.O4), co * co, co * co, Mz, "opm.w_o");
      // dO laid out [i][c][j][d] so both contractions below read it as a plain matrix
      GemmOp g = mk(Mz, co * co, Cz, B(pl.G2), Cz, 0, W("opm.w_o"), co * co, 1, B(pl.dO4), 0);
      g.e.map = OutMap{R, co * R * co, co, co, R * co, 1};
      gemm(g);
      // da[s][(i,c)] = sum_(j,d) b[s][(j,d)] dO[(i,c)][(j,d)]
      GemmOp ga = mk(S, R * co, R * co, at(B(pl.ab4), Mm * co), R * co, 0, B(pl.dO4), R * co, 0, B(pl.dab4), 0);
      ga.e.map = OutMap{1ll << 40, 0, R * 2 * co, co, 2 * co, 1};
      ga.cls = "opm_outer";
      gemm(ga);
      // db[s][(j,d)] = sum_(i,c) a[s][(i,c)] dO[(i,c)][(j,d)]
      GemmOp gb = mk(S, R * co, R * co, B(pl.ab4), R * co, 0, B(pl.dO4), R * co, 1, at(B(pl.dab4), co), 0);
      gb.e.map = OutMap{1ll << 40, 0, R * 2 * co, co, 2 * co, 1};
      gb.cls = "opm_outer";
      gemm(gb);
      ck(row_scale(B(pl.dab4), mm, B(pl.dab4), Mm, (int)(2 * co), bf, s, D("opm.b_ab")));
      dW(B(pl.dab4), 2 * co, 2 * co, B(pl.xm4), Cm, Cm, Mm, "opm.w_ab");
      GemmOp x = mk(Mm, Cm, 2 * co, B(pl.dab4), 2 * co, 0, W("opm.w_ab"), Cm, 1, B(pl.G2), Cm);
      gemm(x);
      lnb(B(pl.G2), B(pl.m3), "opm.ln", dm, dmT, nullptr, Mm, (int)Cm, dm_out, D("msa_trans.b2"));
    }
    // 3. MSA transition
    transition_bwd("msa_trans", B(pl.m2), B(pl.xm3), B(pl.h3), dm, dmT, dmT, Mm, Cm, nullptr, true, D("col.b_o"));
    // 2. MSA column attention (or global column attention)
    if (d.msa_col_mode == EVO_COL_GLOBAL) {
      const int64_t HC = k.HCm, QK = k.QKc;
      dW(dmT, Cm, Cm, B(pl.og2), HC, HC, Mm, "col.w_o");  // col.b_o: added by the MSA transition's LayerNorm backward
      GemmOp g = mk(Mm, HC, Cm, dmT, Cm, 0, W("col.w_o"), HC, 1, B(pl.G2), HC);
      gemm(g);
      ck(global_attn_bwd(global_args(), B(pl.G2), B(pl.G1), nullptr, bf, s));
      dW(B(pl.G1), QK, QK, B(pl.xm2), Cm, Cm, Mm, "col.w_qkvg");
      db(at(B(pl.G1), HC + 2 * k.cm), QK, Mm, HC, "col.b_g");
      GemmOp x = mk(Mm, Cm, QK, B(pl.G1), QK, 0, W("col.w_qkvg"), Cm, 1, B(pl.G2), Cm);
      gemm(x);
    } else {
      attention_bwd(1, "col", B(pl.xm2), B(pl.qkvg2), B(pl.oatt2), B(pl.og2), Bf(pl.lse2), nullptr, mm, dmT, Mm, Cm,
                    true);
    }
    lnb(B(pl.G2), B(pl.m1), "col.ln", dm, dmT, nullptr, Mm, (int)Cm, nullptr, dsc(0) ? nullptr : D("row.b_o"));
    // 1. MSA row attention with pair bias
    {
      const float *sc = dsc(0);
      if (sc) ck(dropout_apply(dmT, sc, nullptr, B(pl.drop_u), Mm, (int)Cm, (int)k.R, 0, bf, s));
      attention_bwd(0, "row", B(pl.xm1), B(pl.qkvg1), B(pl.oatt1), B(pl.og1), Bf(pl.lse1), Bf(pl.bias1), mm,
                    sc ? B(pl.drop_u) : dmT, Mm, Cm, sc == nullptr);
    }
    lnb(B(pl.G2), m0, "row.ln_m", dm, dm_in, nullptr, Mm, (int)Cm);
    pair_bias_bwd("row.w_b", B(pl.xz1), (int)k.Hm, 0, 0);
    lnb(B(pl.G2), z0, "row.ln_z", dz, dz_in, nullptr, Mz, (int)Cz);
  }
};

}  // namespace

size_t workspace_bytes(const evo_dims &d, int mode, bool pair_only) {
  Plan p;
  return make_plan(d, mode, p, pair_only);
}

int block_forward(const evo_dims &d, const float *p32, const bf16 *p16, const void *m_in, const void *z_in,
                  void *m_out, void *z_out, const float *msa_mask, const float *pair_mask, void *ws, size_t ws_bytes,
                  cudaStream_t s, const evo_dropout *dropout) {
  Drv drv(d, p32, p16, ws, EVO_MODE_FWD, s);
  drv.drop = dropout;
  if (ws_bytes < drv.pl.total) return EVO_ERR_WORKSPACE;
  drv.forward(m_in, z_in, m_out, z_out, msa_mask, pair_mask);
  return drv.err == cudaSuccess ? EVO_OK : EVO_ERR_CUDA;
}

int block_forward_infer(const evo_dims &d, const float *p32, const bf16 *p16, const void *m_in, const void *z_in,
                        void *m_out, void *z_out, const float *msa_mask, const float *pair_mask, void *ws,
                        size_t ws_bytes, cudaStream_t s) {
  Drv drv(d, p32, p16, ws, EVO_MODE_INFER, s);
  if (ws_bytes < drv.pl.total) return EVO_ERR_WORKSPACE;
  drv.forward(m_in, z_in, m_out, z_out, msa_mask, pair_mask);
  return drv.err == cudaSuccess ? EVO_OK : EVO_ERR_CUDA;
}

int pair_block_forward(const evo_dims &d, const float *p32, const bf16 *p16, const void *z_in, void *z_out,
                       const float *pair_mask, void *ws, size_t ws_bytes, cudaStream_t s, const evo_dropout *dropout) {
  Drv drv(d, p32, p16, ws, EVO_MODE_FWD, s, true);
  if (ws_bytes < drv.pl.total) return EVO_ERR_WORKSPACE;
  drv.drop = dropout;
  drv.pair_forward(z_in, z_out, pair_mask);
  return drv.err == cudaSuccess ? EVO_OK : EVO_ERR_CUDA;
}

int pair_block_backward(const evo_dims &d, const float *p32, const bf16 *p16, const void *z_in, const float *pair_mask,
                        const void *dz_out, void *dz_in, float *dparams, void *ws, size_t ws_bytes, cudaStream_t s,
                        const evo_dropout *dropout) {
  Drv drv(d, p32, p16, ws, EVO_MODE_BWD, s, true);
  if (ws_bytes < drv.pl.total) return EVO_ERR_WORKSPACE;
  drv.drop = dropout;
  drv.dparams = dparams;
  drv.pair_forward(z_in, nullptr, pair_mask);
  drv.pair_backward(z_in, pair_mask, dz_out, dz_in);
  return drv.err == cudaSuccess ? EVO_OK : EVO_ERR_CUDA;
}

int block_backward(const evo_dims &d, const float *p32, const bf16 *p16, const void *m_in, const void *z_in,
                   const float *msa_mask, const float *pair_mask, const void *dm_out, const void *dz_out, void *dm_in,
                   void *dz_in, float *dparams, void *ws, size_t ws_bytes, cudaStream_t s, const evo_dropout *dropout) {
  Drv drv(d, p32, p16, ws, EVO_MODE_BWD, s);
  drv.drop = dropout;
  if (ws_bytes < drv.pl.total) return EVO_ERR_WORKSPACE;
  drv.dparams = dparams;
  drv.forward(m_in, z_in, nullptr, nullptr, msa_mask, pair_mask);
  drv.backward(m_in, z_in, msa_mask, pair_mask, dm_out, dz_out, dm_in, dz_in);
  return drv.err == cudaSuccess ? EVO_OK : EVO_ERR_CUDA;
}

}  // namespace evo
