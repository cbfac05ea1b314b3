// Host side of the C ABI declared in include/shacsim.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/shacsim.h"
#include "shac_jit.h"
#include "shac_kernels.cuh"

using namespace shac;

struct shac_model {
  int L = 0, nq = 0, nv = 0, na = 0, ntact = 0, nc = 0, nm = 0, nseg = 0, nitems = 0, K = 1, nlev = 0;
  float h = 0, grav[3] = {0, 0, 0}, ke = 0, kd = 0, kt = 0, mu = 0, klim = 0, rc[10] = {0};
  int root_free = 0;
  int height_q = -1, vx_dof = -1;   // reward / termination coordinates (free root: 2 / world vx)
  std::vector<int> parent, jtype, qs, ds, nd, lvl_ptr, lvl_link, ch_ptr, ch_idx, lc_ptr, lc_idx, lm_ptr, lm_idx, dof_link,
      dof_k,
      dof_act, item_link, seg_mus, mus_seg_ptr, anc_mask, chain_tail;
  std::vector<float> axis, jpos, jrot, mass, com, icom, qlo, qhi, arm, damp, gear, item_pos, crad, fmax, rwq, rwqd;
  DevModel layout;   // sizes + scratch offsets (pointers unset)
};

struct Group {
  const shac_model* m;
  int N;
  void* blob = nullptr;      // device copy of the model arrays
  DevModel dev;              // with device pointers
  int lanes = 0;             // batched team size
};

struct shac_batch {
  std::vector<Group> groups;
  int form = SHAC_FORM_BATCHED;
  int h_max = 1;
  int warps_per_cta = 4;
  int64_t q_size = 0, qd_size = 0, act_size = 0, n_envs = 0;
  IOArgs io{};
  DevModel* d_models = nullptr;
  unsigned int* d_flags = nullptr;
  WorkItem* d_items = nullptr;
  int n_items = 0;
  int64_t items_cap = 0;   // capacity of d_items (sum of N_g: one environment per item)
  int device = 0, num_sms = 0;
  // workspace layout (bytes)
  size_t ws_counter = 0, ws_tape = 0, ws_plain = 0, ws_total = 0;
  std::vector<size_t> plain_scratch_off, plain_tape_off, batched_tape_off;
  // window tape (batched): every step's substep records kept by the forward window
  int window_tape = 0;
  size_t ws_step = 0;                    // bytes the step-level calls use (a prefix of the workspace)
  std::vector<size_t> window_tape_off;   // bytes
  std::vector<int64_t> window_tape_step; // floats per step per environment slot
  // model-specialised kernels (shac_batch_specialize): used while group 0 keeps
  // the team size they were built for
  JitKernels spec;
  int spec_lanes = 0;
};

static shac_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? SHAC_OK : SHAC_ERR_CUDA; }

// ------------------------------------------------------------------ model --

static void quat_rot(const float* q, float* R) {
  double x = q[0], y = q[1], z = q[2], w = q[3];
  double n = std::sqrt(x * x + y * y + z * z + w * w);
  x /= n; y /= n; z /= n; w /= n;
  double r[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
                 2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
                 2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)};
  for (int i = 0; i < 9; ++i) R[i] = (float)r[i];
}

static void compute_layout(shac_model* m) {
  DevModel& d = m->layout;
  std::memset(&d, 0, sizeof(d));
  d.L = m->L; d.nq = m->nq; d.nv = m->nv; d.na = m->na; d.ntact = m->ntact; d.nc = m->nc; d.nm = m->nm;
  d.nseg = m->nseg; d.nitems = m->nitems; d.K = m->K; d.nlev = m->nlev; d.h = m->h;
  for (int k = 0; k < 3; ++k) d.grav[k] = m->grav[k];
  d.ke = m->ke; d.kd = m->kd; d.kt = m->kt; d.mu = m->mu; d.klim = m->klim;
  for (int k = 0; k < 10; ++k) d.rc[k] = m->rc[k];
  d.root_free = m->root_free;
  d.height_q = m->height_q;
  d.vx_dof = m->vx_dof;
  const int L = m->L, nv = m->nv, ni = m->nitems;
  int o = 0;
  auto take = [&](int& off, int n) { off = o; o += n; };
  // substep record: the start state and every forward intermediate the reverse
  // pass reads (per link: pose, spatial inertia, velocity, external wrench)
  take(d.o_Q, m->nq); take(d.o_QD, nv); take(d.o_LR, LREC * L);
  take(d.o_S, 6 * nv); take(d.o_IT, 7 * ni);
  take(d.o_M, nv * nv); take(d.o_LD, nv); take(d.o_QDD, nv);
  o = (o + 3) / 4 * 4;   // records are copied 16 bytes at a time
  d.rec_floats = o;
  take(d.o_ACT, m->na); take(d.o_QB, m->nq); take(d.o_QDB, nv); take(d.o_ACTB, m->na);
  take(d.o_QC, m->nq); take(d.o_QDC, nv); take(d.o_LW, LWORK * L);
  take(d.o_B, nv); take(d.o_T, nv);
  take(d.o_LAM, nv); take(d.o_ITB, 10 * ni);
  take(d.o_SEGA, m->nseg);
  // free root: its six DOFs' reverse terms (velocity cotangent sums 6, then
  // one rotation-column share of 3 per DOF)
  take(d.o_RDB, m->root_free ? 18 : 0);   // the free root's six DOF shares of its rotation cotangent
  // partial muscle sums of (link, part) slots: at most max(32, L) slots (parts
  // = lanes / links when a team has at least two lanes per link, else 1),
  // 6 floats forward, 12 in reverse
  take(d.o_MW, m->nseg > 0 ? std::max(32, L) * 12 : 0);
  d.env_floats = o;
}

extern "C" shac_status shac_model_create(const shac_model_desc* dsc, shac_model** out) {
  if (!dsc || !out) return SHAC_ERR_INVALID_ARG;
  *out = nullptr;
  const int L = dsc->n_links;
  if (L <= 0) return SHAC_ERR_MODEL;
  if (L > MAX_LINKS) return SHAC_ERR_CAPACITY;
  if (!dsc->parent || !dsc->joint_type || !dsc->joint_axis || !dsc->joint_pos || !dsc->joint_quat || !dsc->mass ||
      !dsc->com || !dsc->inertia)
    return SHAC_ERR_INVALID_ARG;
  if (dsc->substeps < 1 || !(dsc->dt > 0.f)) return SHAC_ERR_INVALID_ARG;
  shac_model* m = new (std::nothrow) shac_model();
  if (!m) return SHAC_ERR_INVALID_ARG;
  m->L = L;
  m->parent.assign(dsc->parent, dsc->parent + L);
  m->jtype.assign(dsc->joint_type, dsc->joint_type + L);
  int nq = 0, nv = 0;
  for (int i = 0; i < L; ++i) {
    const int p = m->parent[i], t = m->jtype[i];
    if (p < -1 || p >= i || t < 0 || t > 3 || (t == J_FREE && (p != -1 || i != 0))) { delete m; return SHAC_ERR_MODEL; }
    m->qs.push_back(nq);
    m->ds.push_back(nv);
    const int ndof = t == J_FREE ? 6 : (t == J_FIXED ? 0 : 1);
    m->nd.push_back(ndof);
    nq += t == J_FREE ? 7 : ndof;
    nv += ndof;
  }
  if (nv < 1) { delete m; return SHAC_ERR_MODEL; }
  if (nv > MAX_DOF) { delete m; return SHAC_ERR_CAPACITY; }
  m->nq = nq; m->nv = nv;
  m->root_free = m->jtype[0] == J_FREE;
  if (m->root_free) {
    m->height_q = 2;   // root origin height; the forward velocity is the root's world vx
  } else {
    if (dsc->height_q < -1 || dsc->height_q >= nq || dsc->vx_dof < -1 || dsc->vx_dof >= nv) {
      delete m;
      return SHAC_ERR_MODEL;
    }
    m->height_q = dsc->height_q;
    m->vx_dof = dsc->vx_dof;
  }
  for (int i = 0; i < L; ++i) {
    float a[3] = {dsc->joint_axis[3 * i], dsc->joint_axis[3 * i + 1], dsc->joint_axis[3 * i + 2]};
    float n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if ((m->jtype[i] == J_REV || m->jtype[i] == J_PRIS) && !(n > 0.f)) { delete m; return SHAC_ERR_MODEL; }
    for (int k = 0; k < 3; ++k) m->axis.push_back(n > 0.f ? a[k] / n : 0.f);
    for (int k = 0; k < 3; ++k) m->jpos.push_back(dsc->joint_pos[3 * i + k]);
    float R[9];
    quat_rot(dsc->joint_quat + 4 * i, R);
    for (int k = 0; k < 9; ++k) m->jrot.push_back(R[k]);
    m->mass.push_back(dsc->mass[i]);
    for (int k = 0; k < 3; ++k) m->com.push_back(dsc->com[3 * i + k]);
    for (int k = 0; k < 6; ++k) m->icom.push_back(dsc->inertia[6 * i + k]);
  }
  // children lists
  m->ch_ptr.assign(L + 1, 0);
  for (int i = 0; i < L; ++i) {
    m->ch_ptr[i] = (int)m->ch_idx.size();
    for (int c = i + 1; c < L; ++c)
      if (m->parent[c] == i) m->ch_idx.push_back(c);
  }
  m->ch_ptr[L] = (int)m->ch_idx.size();
  // Chains: maximal runs of links in which every link but the last has exactly
  // one child; a chain is swept by one lane (parent before child), so tree
  // sweeps need one team barrier per chain level instead of per link depth.
  std::vector<int> head(L), cdepth(L, 0);
  m->chain_tail.assign(L, -1);
  int maxd = 0;
  for (int i = 0; i < L; ++i) {
    const int p = m->parent[i];
    const bool cont = p >= 0 && m->ch_ptr[p + 1] - m->ch_ptr[p] == 1;
    head[i] = cont ? head[p] : i;
    cdepth[i] = p < 0 ? 0 : (cont ? cdepth[p] : cdepth[p] + 1);
    maxd = std::max(maxd, cdepth[i]);
  }
  for (int i = 0; i < L; ++i) m->chain_tail[head[i]] = i;   // links are numbered parent first
  m->nlev = maxd + 1;
  m->lvl_ptr.assign(m->nlev + 1, 0);
  for (int l = 0; l < m->nlev; ++l) {
    m->lvl_ptr[l] = (int)m->lvl_link.size();
    for (int i = 0; i < L; ++i)
      if (head[i] == i && cdepth[i] == l) m->lvl_link.push_back(i);
  }
  m->lvl_ptr[m->nlev] = (int)m->lvl_link.size();
  // dofs
  for (int i = 0; i < L; ++i)
    for (int k = 0; k < m->nd[i]; ++k) { m->dof_link.push_back(i); m->dof_k.push_back(k); }
  for (int a = 0; a < nv; ++a) {
    unsigned mask = 0u;
    for (int j = m->dof_link[a]; j >= 0; j = m->parent[j])
      for (int b = m->ds[j]; b < m->ds[j] + m->nd[j]; ++b)
        if (b <= a) mask |= 1u << b;
    m->anc_mask.push_back((int)mask);
  }
  if (!dsc->q_lower || !dsc->q_upper || !dsc->armature || !dsc->joint_damping) { delete m; return SHAC_ERR_INVALID_ARG; }
  m->qlo.assign(dsc->q_lower, dsc->q_lower + nv);
  m->qhi.assign(dsc->q_upper, dsc->q_upper + nv);
  m->arm.assign(dsc->armature, dsc->armature + nv);
  m->damp.assign(dsc->joint_damping, dsc->joint_damping + nv);
  m->klim = dsc->k_limit;
  m->ntact = dsc->n_tact;
  if (m->ntact < 0 || (m->ntact > 0 && (!dsc->act_dof || !dsc->act_gear))) { delete m; return SHAC_ERR_INVALID_ARG; }
  m->dof_act.assign(nv, -1);
  m->gear.assign(nv, 0.f);
  for (int k = 0; k < m->ntact; ++k) {
    const int d = dsc->act_dof[k];
    if (d < 0 || d >= nv || m->dof_act[d] >= 0) { delete m; return SHAC_ERR_MODEL; }
    m->dof_act[d] = k;
    m->gear[d] = dsc->act_gear[k];
  }
  // contacts
  m->nc = dsc->n_contacts;
  if (m->nc < 0) { delete m; return SHAC_ERR_INVALID_ARG; }
  if (m->nc > MAX_CONTACTS) { delete m; return SHAC_ERR_CAPACITY; }
  if (m->nc > 0 && (!dsc->contact_link || !dsc->contact_pos || !dsc->contact_radius)) { delete m; return SHAC_ERR_INVALID_ARG; }
  for (int c = 0; c < m->nc; ++c) {
    const int l = dsc->contact_link[c];
    if (l < 0 || l >= L) { delete m; return SHAC_ERR_MODEL; }
    m->item_link.push_back(l);
    for (int k = 0; k < 3; ++k) m->item_pos.push_back(dsc->contact_pos[3 * c + k]);
    m->crad.push_back(dsc->contact_radius[c]);
  }
  // muscles -> segments -> two items each
  m->nm = dsc->n_muscles;
  if (m->nm < 0 || (m->nm > 0 && (!dsc->muscle_ptr || !dsc->via_link || !dsc->via_pos || !dsc->muscle_fmax))) {
    delete m; return SHAC_ERR_INVALID_ARG;
  }
  m->mus_seg_ptr.assign(m->nm + 1, 0);
  for (int k = 0; k < m->nm; ++k) {
    const int v0 = dsc->muscle_ptr[k], v1 = dsc->muscle_ptr[k + 1];
    if (v1 - v0 < 2) { delete m; return SHAC_ERR_MODEL; }
    m->mus_seg_ptr[k] = m->nseg;
    for (int v = v0; v + 1 < v1; ++v) {
      const int la = dsc->via_link[v], lb = dsc->via_link[v + 1];
      if (la < 0 || la >= L || lb < 0 || lb >= L) { delete m; return SHAC_ERR_MODEL; }
      m->item_link.push_back(la);
      for (int j = 0; j < 3; ++j) m->item_pos.push_back(dsc->via_pos[3 * v + j]);
      m->item_link.push_back(lb);
      for (int j = 0; j < 3; ++j) m->item_pos.push_back(dsc->via_pos[3 * (v + 1) + j]);
      m->seg_mus.push_back(k);
      m->nseg++;
    }
    m->fmax.push_back(dsc->muscle_fmax[k]);
  }
  m->mus_seg_ptr[m->nm] = m->nseg;
  m->nitems = m->nc + 2 * m->nseg;
  // per-link lists of the contact items and of the muscle via-point items
  m->lc_ptr.assign(L + 1, 0);
  m->lm_ptr.assign(L + 1, 0);
  for (int i = 0; i < L; ++i) {
    m->lc_ptr[i] = (int)m->lc_idx.size();
    m->lm_ptr[i] = (int)m->lm_idx.size();
    for (int e = 0; e < m->nitems; ++e)
      if (m->item_link[e] == i) (e < m->nc ? m->lc_idx : m->lm_idx).push_back(e);
  }
  m->lc_ptr[L] = (int)m->lc_idx.size();
  m->lm_ptr[L] = (int)m->lm_idx.size();
  m->na = m->ntact + m->nm;
  m->K = dsc->substeps;
  m->h = (float)((double)dsc->dt / dsc->substeps);
  for (int k = 0; k < 3; ++k) m->grav[k] = dsc->gravity[k];
  m->ke = dsc->ke; m->kd = dsc->kd; m->kt = dsc->kt; m->mu = dsc->mu;
  if (!dsc->rw_q || !dsc->rw_qd) { delete m; return SHAC_ERR_INVALID_ARG; }
  m->rwq.assign(dsc->rw_q, dsc->rw_q + nq);
  m->rwqd.assign(dsc->rw_qd, dsc->rw_qd + nv);
  for (int k = 0; k < 10; ++k) m->rc[k] = dsc->reward_coef[k];
  compute_layout(m);
  *out = m;
  return SHAC_OK;
}

extern "C" void shac_model_destroy(shac_model* m) { delete m; }

extern "C" void shac_model_dims(const shac_model* m, int32_t* nq, int32_t* nv, int32_t* na) {
  if (!m) return;
  if (nq) *nq = m->nq;
  if (nv) *nv = m->nv;
  if (na) *na = m->na;
}

// Upload one model's arrays into a single device blob and point a DevModel at it.
static shac_status upload_model(const shac_model* m, Group& g) {
  std::vector<int> iblob;
  std::vector<float> fblob;
  std::vector<std::pair<const int**, size_t>> ifix;
  std::vector<std::pair<const float**, size_t>> ffix;
  DevModel& d = g.dev;
  d = m->layout;
  auto addi = [&](const int** dst, const std::vector<int>& v) {
    ifix.push_back({dst, iblob.size()});
    iblob.insert(iblob.end(), v.begin(), v.end());
    iblob.push_back(0);   // never empty
  };
  auto addf = [&](const float** dst, const std::vector<float>& v) {
    ffix.push_back({dst, fblob.size()});
    fblob.insert(fblob.end(), v.begin(), v.end());
    fblob.push_back(0.f);
  };
  addi(&d.parent, m->parent); addi(&d.jtype, m->jtype); addi(&d.qs, m->qs); addi(&d.ds, m->ds); addi(&d.nd, m->nd);
  addi(&d.lvl_ptr, m->lvl_ptr); addi(&d.lvl_link, m->lvl_link); addi(&d.chain_tail, m->chain_tail); addi(&d.ch_ptr, m->ch_ptr); addi(&d.ch_idx, m->ch_idx);
  addi(&d.lc_ptr, m->lc_ptr); addi(&d.lc_idx, m->lc_idx); addi(&d.lm_ptr, m->lm_ptr); addi(&d.lm_idx, m->lm_idx);
  addi(&d.dof_link, m->dof_link); addi(&d.dof_k, m->dof_k);
  addi(&d.dof_act, m->dof_act); addi(&d.item_link, m->item_link); addi(&d.seg_mus, m->seg_mus);
  addi(&d.mus_seg_ptr, m->mus_seg_ptr);
  {
    const int* tmp = nullptr;
    addi(&tmp, m->anc_mask);
    ifix.back().first = reinterpret_cast<const int**>(&d.anc_mask);
  }
  addf(&d.axis, m->axis); addf(&d.jpos, m->jpos); addf(&d.jrot, m->jrot); addf(&d.mass, m->mass); addf(&d.com, m->com);
  addf(&d.icom, m->icom); addf(&d.qlo, m->qlo); addf(&d.qhi, m->qhi); addf(&d.arm, m->arm); addf(&d.damp, m->damp);
  addf(&d.gear, m->gear); addf(&d.item_pos, m->item_pos); addf(&d.crad, m->crad); addf(&d.fmax, m->fmax);
  addf(&d.rwq, m->rwq); addf(&d.rwqd, m->rwqd);
  const size_t ibytes = ((iblob.size() * sizeof(int) + 255) / 256) * 256;
  const size_t bytes = ibytes + fblob.size() * sizeof(float);
  char* dev = nullptr;
  if (cudaMalloc(&dev, bytes) != cudaSuccess) return SHAC_ERR_CUDA;
  std::vector<char> host(bytes, 0);
  std::memcpy(host.data(), iblob.data(), iblob.size() * sizeof(int));
  std::memcpy(host.data() + ibytes, fblob.data(), fblob.size() * sizeof(float));
  if (cudaMemcpy(dev, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) { cudaFree(dev); return SHAC_ERR_CUDA; }
  for (auto& f : ifix) *f.first = reinterpret_cast<const int*>(dev) + f.second;
  for (auto& f : ffix) *f.first = reinterpret_cast<const float*>(dev + ibytes) + f.second;
  g.blob = dev;
  return SHAC_OK;
}

static int default_lanes(const shac_model* m) {
  const int par = std::max(m->nv, m->L);
  if (par <= 2) return 2;
  if (par <= 4) return 4;
  if (par <= 8) return 8;
  if (par <= 16) return 16;
  return 32;
}

// Register row capacity of the batched dense path: the smallest of the device
// instantiations (2, 4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32 rows) that holds
// nv rows, one padded row per lane, when the team has that many lanes; 0
// selects the shared-memory form.
static int dense_class(int nv, int lanes) {
  static const int sizes[] = {2, 4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32};
  for (int nm : sizes)
    if (nm >= nv) return nm <= lanes ? nm : 0;
  return 0;
}

// Shared floats per environment: padded so that every environment's scratch
// starts 16-byte aligned (records move 16 bytes at a time) and the 32 / lanes
// teams of a warp start spread over the 32 banks (lanes apart, at least 4).
static int env_stride(const shac_model* m, int lanes) {
  return ((m->layout.env_floats + 31) / 32) * 32 + (lanes >= 4 ? lanes % 32 : 4);
}

static size_t batched_smem_warp_floats(const shac_batch* b) {
  size_t per_warp = 0;
  for (const Group& g : b->groups) {
    if (g.N == 0) continue;
    per_warp = std::max(per_warp, (size_t)(32 / g.lanes) * env_stride(g.m, g.lanes));
  }
  return per_warp;
}

// Dynamic shared memory available to one CTA (227 KB per block on sm_103,
// minus the kernels' static shared memory and a margin).
constexpr size_t SMEM_BLOCK_LIMIT = 227 * 1024 - 8 * 1024;

// Warps per CTA actually launched: the requested count, reduced until the
// per-warp scratch fits in one CTA's shared memory (0 if one warp does not fit).
static int batched_warps(const shac_batch* b) {
  const size_t per_warp = batched_smem_warp_floats(b) * sizeof(float);
  int W = b->warps_per_cta;
  while (W > 0 && (size_t)W * per_warp > SMEM_BLOCK_LIMIT) --W;
  return W;
}

// Work items sorted by per-warp cost (largest first) so the dynamic schedule
// finishes the long items early.
static shac_status build_items(shac_batch* b) {
  std::vector<std::pair<double, WorkItem>> items;
  for (int gi = 0; gi < (int)b->groups.size(); ++gi) {
    const Group& g = b->groups[gi];
    const int per = 32 / g.lanes;
    const shac_model* m = g.m;
    const double cost = (double)m->K * ((double)m->nv * m->nv + 40.0 * m->L + 20.0 * m->nitems) * g.lanes / 32.0 * per;
    for (int e = 0; e < g.N; e += per) items.push_back({cost, WorkItem{gi, e, std::min(per, g.N - e)}});
  }
  std::stable_sort(items.begin(), items.end(), [](const auto& a, const auto& c) { return a.first > c.first; });
  std::vector<WorkItem> h;
  for (auto& p : items) h.push_back(p.second);
  // the item buffer is allocated once, in shac_batch_create, for the largest
  // item count (one environment per item)
  if ((int64_t)h.size() > b->items_cap) return SHAC_ERR_CAPACITY;
  b->n_items = (int)h.size();
  if (h.empty()) return SHAC_OK;
  return cuda_ok(cudaMemcpy(b->d_items, h.data(), h.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
}

static void compute_workspace(shac_batch* b) {
  size_t off = 256;   // [0, 256): work counter
  b->ws_counter = 0;
  b->plain_scratch_off.assign(b->groups.size(), 0);
  b->plain_tape_off.assign(b->groups.size(), 0);
  b->batched_tape_off.assign(b->groups.size(), 0);
  auto align = [](size_t x) { return (x + 255) / 256 * 256; };
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const Group& g = b->groups[gi];
    const shac_model* m = g.m;
    const size_t S = (size_t)(m->nq + m->nv) * m->K;
    const size_t REC = (size_t)m->layout.rec_floats * m->K;
    if (b->form == SHAC_FORM_PLAIN) {
      b->plain_scratch_off[gi] = off;
      off = align(off + (size_t)m->layout.env_floats * g.N * sizeof(float));
      b->plain_tape_off[gi] = off;
      off = align(off + S * g.N * sizeof(float));
    } else {
      b->batched_tape_off[gi] = off;   // one step's substep records per environment slot
      off = align(off + REC * (size_t)(g.N + 31) * sizeof(float));
    }
  }
  b->ws_step = off;
  b->window_tape_off.assign(b->groups.size(), 0);
  b->window_tape_step.assign(b->groups.size(), 0);
  if (b->form == SHAC_FORM_BATCHED && b->window_tape) {
    // h_max steps x (K records + post-step q, qd) per environment slot
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
      const shac_model* m = b->groups[gi].m;
      b->window_tape_step[gi] = ((int64_t)m->layout.rec_floats * m->K + m->nq + m->nv + 3) / 4 * 4;
      b->window_tape_off[gi] = off;
      off = align(off + (size_t)b->window_tape_step[gi] * b->h_max * (size_t)(b->groups[gi].N + 31) * sizeof(float));
    }
  }
  b->ws_total = off;
}

extern "C" shac_status shac_batch_create(const shac_model* const* models, const int32_t* n_envs, int32_t n_groups,
                                         int32_t form, int32_t window_h_max, shac_batch** out) {
  if (!models || !n_envs || !out || n_groups < 1 || n_groups > MAX_GROUPS || window_h_max < 1) return SHAC_ERR_INVALID_ARG;
  if (form != SHAC_FORM_PLAIN && form != SHAC_FORM_BATCHED) return SHAC_ERR_INVALID_ARG;
  *out = nullptr;
  shac_batch* b = new (std::nothrow) shac_batch();
  if (!b) return SHAC_ERR_INVALID_ARG;
  b->form = form;
  b->h_max = window_h_max;
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
    delete b;
    return SHAC_ERR_CUDA;
  }
  b->io.n_groups = n_groups;
  for (int gi = 0; gi < n_groups; ++gi) {
    if (!models[gi] || n_envs[gi] < 0) { shac_batch_destroy(b); return SHAC_ERR_INVALID_ARG; }
    Group g;
    g.m = models[gi];
    g.N = n_envs[gi];
    g.lanes = default_lanes(g.m);
    shac_status st = upload_model(g.m, g);
    if (st != SHAC_OK) { shac_batch_destroy(b); return st; }
    GroupIO& io = b->io.g[gi];
    io.N = g.N;
    io.q_off = b->q_size; io.qd_off = b->qd_size; io.act_off = b->act_size; io.env_off = b->n_envs;
    b->q_size += (int64_t)g.m->nq * g.N;
    b->qd_size += (int64_t)g.m->nv * g.N;
    b->act_size += (int64_t)g.m->na * g.N;
    b->n_envs += g.N;
    b->groups.push_back(g);
  }
  b->io.q_size = b->q_size; b->io.qd_size = b->qd_size; b->io.act_size = b->act_size; b->io.n_envs = b->n_envs;
  std::vector<DevModel> dm;
  for (auto& g : b->groups) dm.push_back(g.dev);
  if (cudaMalloc(&b->d_models, dm.size() * sizeof(DevModel)) != cudaSuccess ||
      cudaMemcpy(b->d_models, dm.data(), dm.size() * sizeof(DevModel), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMalloc(&b->d_flags, sizeof(unsigned int)) != cudaSuccess ||
      cudaMemset(b->d_flags, 0, sizeof(unsigned int)) != cudaSuccess) {
    shac_batch_destroy(b);
    return SHAC_ERR_CUDA;
  }
  b->items_cap = std::max<int64_t>(1, b->n_envs);
  if (cudaMalloc(&b->d_items, (size_t)b->items_cap * sizeof(WorkItem)) != cudaSuccess) {
    shac_batch_destroy(b);
    return SHAC_ERR_CUDA;
  }
  shac_status st = build_items(b);
  if (st != SHAC_OK) { shac_batch_destroy(b); return st; }
  compute_workspace(b);
  *out = b;
  return SHAC_OK;
}

extern "C" void shac_batch_destroy(shac_batch* b) {
  if (!b) return;
  for (auto& g : b->groups)
    if (g.blob) cudaFree(g.blob);
  if (b->d_models) cudaFree(b->d_models);
  if (b->d_flags) cudaFree(b->d_flags);
  if (b->d_items) cudaFree(b->d_items);
  delete b;
}

extern "C" void shac_batch_dims(const shac_batch* b, int64_t* q_size, int64_t* qd_size, int64_t* act_size,
                                int64_t* n_envs) {
  if (!b) return;
  if (q_size) *q_size = b->q_size;
  if (qd_size) *qd_size = b->qd_size;
  if (act_size) *act_size = b->act_size;
  if (n_envs) *n_envs = b->n_envs;
}

extern "C" size_t shac_batch_workspace_bytes(const shac_batch* b) { return b ? b->ws_total : 0; }

extern "C" shac_status shac_batch_set_launch(shac_batch* b, int32_t group, int32_t lanes, int32_t warps) {
  if (!b || group < -1 || group >= (int)b->groups.size()) return SHAC_ERR_INVALID_ARG;
  if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32)
    return SHAC_ERR_INVALID_ARG;
  if (warps < 0 || warps > 8) return SHAC_ERR_INVALID_ARG;
  for (int gi = 0; gi < (int)b->groups.size(); ++gi) {
    if (group >= 0 && gi != group) continue;
    b->groups[gi].lanes = lanes == 0 ? default_lanes(b->groups[gi].m) : lanes;
  }
  if (warps > 0) b->warps_per_cta = warps;
  return build_items(b);
}

extern "C" shac_status shac_batch_set_window_tape(shac_batch* b, int32_t keep) {
  if (!b || (keep != 0 && keep != 1)) return SHAC_ERR_INVALID_ARG;
  if (keep && b->form != SHAC_FORM_BATCHED) return SHAC_ERR_UNSUPPORTED;
  b->window_tape = keep;
  compute_workspace(b);
  return SHAC_OK;
}

extern "C" shac_status shac_batch_specialize(shac_batch* b, int32_t enable) {
  if (!b || (enable != 0 && enable != 1)) return SHAC_ERR_INVALID_ARG;
  if (!enable) {
    b->spec = JitKernels{};
    b->spec_lanes = 0;
    return SHAC_OK;
  }
  if (b->form != SHAC_FORM_BATCHED || b->groups.size() != 1) return SHAC_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SHAC_ERR_CUDA;
  if (dev != b->device) return SHAC_ERR_INVALID_ARG;
  const Group& g = b->groups[0];
  JitKernels k;
  const shac_status st = jit_kernels(b->device, g.m->layout, g.m->parent, g.lanes, dense_class(g.m->nv, g.lanes),
                                     env_stride(g.m, g.lanes), &k, nullptr);
  if (st != SHAC_OK) return st;
  b->spec = k;
  b->spec_lanes = g.lanes;
  return SHAC_OK;
}

extern "C" shac_status shac_batch_get_launch(const shac_batch* b, int32_t group, int32_t* lanes, int32_t* warps) {
  if (!b || group < 0 || group >= (int)b->groups.size()) return SHAC_ERR_INVALID_ARG;
  if (lanes) *lanes = b->groups[group].lanes;
  if (warps) *warps = b->form == SHAC_FORM_BATCHED ? batched_warps(b) : b->warps_per_cta;
  return SHAC_OK;
}

// ------------------------------------------------------------- execution --

static PlainGroup plain_group(const shac_batch* b, int gi, void* ws) {
  PlainGroup p;
  p.M = b->groups[gi].dev;
  p.N = b->groups[gi].N;
  p.ws = reinterpret_cast<float*>(static_cast<char*>(ws) + b->plain_scratch_off[gi]);
  p.tape = reinterpret_cast<float*>(static_cast<char*>(ws) + b->plain_tape_off[gi]);
  return p;
}

static shac_status batched_launch(shac_batch* b, BatchedArgs& a, void* ws, cudaStream_t s, bool adjoint,
                                  bool window = false) {
  a.models = b->d_models;
  a.n_groups = (int)b->groups.size();
  a.io = b->io;
  for (int gi = 0; gi < a.n_groups; ++gi) {
    a.lanes[gi] = b->groups[gi].lanes;
    a.env_stride[gi] = env_stride(b->groups[gi].m, b->groups[gi].lanes);
    a.dense_nm[gi] = dense_class(b->groups[gi].m->nv, b->groups[gi].lanes);
  }
  a.smem_warp_floats = (int)batched_smem_warp_floats(b);
  a.items = b->d_items;
  a.n_items = b->n_items;
  a.counter = reinterpret_cast<int*>(static_cast<char*>(ws) + b->ws_counter);
  a.tape = reinterpret_cast<float*>(ws);
  for (int gi = 0; gi < a.n_groups; ++gi) a.tape_off[gi] = (int64_t)(b->batched_tape_off[gi] / sizeof(float));
  if (window && b->window_tape) {
    a.tape_window = 1;
    a.tape_hmax = b->h_max;
    for (int gi = 0; gi < a.n_groups; ++gi) {
      a.tape_off[gi] = (int64_t)(b->window_tape_off[gi] / sizeof(float));
      a.tape_step[gi] = b->window_tape_step[gi];
    }
  }
  a.flags = b->d_flags;
  if (b->n_items == 0) return SHAC_OK;
  const int W = batched_warps(b);
  if (W < 1) return SHAC_ERR_CAPACITY;
  const size_t smem = (size_t)W * a.smem_warp_floats * sizeof(float);
  const int block = 32 * W;
  // the model-specialised kernels while the launch shape is the one they were built for
  const void* spec = nullptr;
  if (b->spec.key != 0u && b->spec_lanes == b->groups[0].lanes) {
    spec = adjoint ? b->spec.adj : b->spec.fwd;
    a.spec_key = b->spec.key;
  }
  // Static plus dynamic shared memory above 48 KB needs the opt-in attribute;
  // the kernels' static part (the model table) is under 8 KB.
  if (smem > 40 * 1024) {
    const cudaError_t e = spec ? cudaFuncSetAttribute(spec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                               : batched_set_smem_limit(smem);
    if (e != cudaSuccess) return SHAC_ERR_CAPACITY;
  }
  int occ = 0;
  const cudaError_t oe = spec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spec, block, smem)
                              : batched_occupancy(&occ, block, smem, adjoint);
  if (oe != cudaSuccess) return SHAC_ERR_CUDA;
  if (occ < 1) return SHAC_ERR_CAPACITY;
  const int grid = std::max(1, std::min(b->num_sms * occ, (b->n_items + W - 1) / W));
  if (cudaMemsetAsync(a.counter, 0, sizeof(int), s) != cudaSuccess) return SHAC_ERR_CUDA;
  if (spec) {
    void* args[] = {&a};
    return cuda_ok(cudaLaunchKernel(spec, dim3(grid), dim3(block), args, smem, s));
  }
  if (adjoint) launch_batched_adjoint(a, grid, block, smem, s);
  else launch_batched_forward(a, grid, block, smem, s);
  return cuda_ok(cudaGetLastError());
}

// Episodic-window arguments (early termination with reset); batched form only.
struct Episodic {
  const float* q_reset = nullptr;
  const float* qd_reset = nullptr;
  const float* term_height = nullptr;   // host [n_groups]
  const int32_t* max_ep = nullptr;      // host [n_groups]
  int* ep_step = nullptr;
  unsigned char* done = nullptr;
  const unsigned char* done_in = nullptr;
};

static void set_episodic(const shac_batch* b, BatchedArgs& a, const Episodic* ep) {
  if (!ep) return;
  a.q_reset = ep->q_reset; a.qd_reset = ep->qd_reset;
  for (int gi = 0; gi < (int)b->groups.size(); ++gi) {
    a.term_h[gi] = ep->term_height ? ep->term_height[gi] : -INFINITY;
    a.max_ep[gi] = ep->max_ep ? ep->max_ep[gi] : 0;
  }
  a.ep_step = ep->ep_step; a.done = ep->done; a.done_in = ep->done_in;
}

static shac_status run_forward(shac_batch* b, cudaStream_t s, void* ws, int h, const float* q0, const float* qd0,
                               const float* act, float* q_out, float* qd_out, float* reward, float* q_copy0,
                               float* qd_copy0, const Episodic* ep = nullptr, bool window = false) {
  if (b->form == SHAC_FORM_BATCHED) {
    BatchedArgs a{};
    a.h = h;
    a.q_in = q0; a.qd_in = qd0; a.act = act;
    a.q_out = q_out; a.qd_out = qd_out; a.reward = reward;
    a.q_copy0 = q_copy0; a.qd_copy0 = qd_copy0;
    set_episodic(b, a, ep);
    return batched_launch(b, a, ws, s, false, window);
  }
  if (ep) return SHAC_ERR_UNSUPPORTED;
  if (q_copy0) {
    if (cudaMemcpyAsync(q_copy0, q0, b->q_size * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(qd_copy0, qd0, b->qd_size * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return SHAC_ERR_CUDA;
  }
  for (int gi = 0; gi < (int)b->groups.size(); ++gi) {
    if (b->groups[gi].N == 0) continue;
    PlainGroup p = plain_group(b, gi, ws);
    const GroupIO& io = b->io.g[gi];
    launch_plain_load(p, q0, qd0, nullptr, io.q_off, io.qd_off, 0, s);
    for (int t = 0; t < h; ++t) {
      launch_plain_load(p, nullptr, nullptr, act + (size_t)t * b->act_size, 0, 0, io.act_off, s);
      for (int k = 0; k < p.M.K; ++k)
        for (int stg = PS_KIN; stg <= PS_INTEGRATE; ++stg) launch_plain_stage(p, stg, s);
      launch_plain_store(p, q_out + (size_t)t * b->q_size, qd_out + (size_t)t * b->qd_size,
                         reward + (size_t)t * b->n_envs, io.q_off, io.qd_off, io.env_off, b->d_flags, s);
    }
  }
  return cuda_ok(cudaGetLastError());
}

// Reverse over h steps.  qtb/qdtb: optional cotangents of checkpoints 0..h-1
// ([h][..]); qT_bar/qdT_bar: cotangent of the final state.
static shac_status run_adjoint(shac_batch* b, cudaStream_t s, void* ws, int h, const float* q_traj,
                               const float* qd_traj, const float* act, const float* reward_bar, const float* qtb,
                               const float* qdtb, const float* qT_bar, const float* qdT_bar, float* q0_bar,
                               float* qd0_bar, float* act_bar, const Episodic* ep = nullptr, bool window = false) {
  if (b->form == SHAC_FORM_BATCHED) {
    BatchedArgs a{};
    a.h = h;
    a.q_traj = q_traj; a.qd_traj = qd_traj; a.act = act; a.reward_bar = reward_bar;
    a.qT_bar = qT_bar; a.qdT_bar = qdT_bar; a.qtb = qtb; a.qdtb = qdtb;
    a.q0_bar = q0_bar; a.qd0_bar = qd0_bar; a.act_bar = act_bar;
    set_episodic(b, a, ep);
    return batched_launch(b, a, ws, s, true, window);
  }
  if (ep) return SHAC_ERR_UNSUPPORTED;
  for (int gi = 0; gi < (int)b->groups.size(); ++gi) {
    if (b->groups[gi].N == 0) continue;
    PlainGroup p = plain_group(b, gi, ws);
    const GroupIO& io = b->io.g[gi];
    for (int t = h - 1; t >= 0; --t) {
      launch_plain_load(p, q_traj + (size_t)t * b->q_size, qd_traj + (size_t)t * b->qd_size,
                        act + (size_t)t * b->act_size, io.q_off, io.qd_off, io.act_off, s);
      for (int k = 0; k < p.M.K; ++k) {
        launch_plain_tape(p, k, true, s);
        for (int stg = PS_KIN; stg <= PS_INTEGRATE; ++stg) launch_plain_stage(p, stg, s);
      }
      const bool last = t == h - 1;
      const float* qa = last ? qT_bar : (qtb ? qtb + (size_t)(t + 1) * b->q_size : nullptr);
      const float* qda = last ? qdT_bar : (qdtb ? qdtb + (size_t)(t + 1) * b->qd_size : nullptr);
      launch_plain_adj_begin(p, qa, qda, reward_bar + (size_t)t * b->n_envs, io.q_off, io.qd_off, io.env_off,
                             last ? 1 : 0, s);
      for (int k = p.M.K - 1; k >= 0; --k) {
        launch_plain_tape(p, k, false, s);
        for (int stg = PS_KIN; stg <= PS_SOLVE; ++stg) launch_plain_stage(p, stg, s);
        launch_plain_stage(p, PS_ADJ_INTEGRATE, s);
        launch_plain_stage(p, PS_ADJ_DYN, s);
      }
      launch_plain_adj_store_act(p, act_bar + (size_t)t * b->act_size, io.act_off, s);
    }
    launch_plain_adj_store_state(p, q0_bar, qd0_bar, qtb, qdtb, io.q_off, io.qd_off, s);
  }
  return cuda_ok(cudaGetLastError());
}

static bool aligned_ws(const shac_batch* b, const void* ws) {
  return ws != nullptr && (reinterpret_cast<uintptr_t>(ws) % 256) == 0 && b->ws_total > 0;
}

extern "C" shac_status shac_step(shac_batch* b, void* stream, void* ws, const float* q, const float* qd,
                                 const float* act, float* q_next, float* qd_next, float* reward) {
  if (!b || !aligned_ws(b, ws) || !q || !qd || !act || !q_next || !qd_next || !reward) return SHAC_ERR_INVALID_ARG;
  return run_forward(b, (cudaStream_t)stream, ws, 1, q, qd, act, q_next, qd_next, reward, nullptr, nullptr);
}

extern "C" shac_status shac_step_adjoint(shac_batch* b, void* stream, void* ws, const float* q, const float* qd,
                                         const float* act, const float* q_next_bar, const float* qd_next_bar,
                                         const float* reward_bar, float* q_bar, float* qd_bar, float* act_bar) {
  if (!b || !aligned_ws(b, ws) || !q || !qd || !act || !q_next_bar || !qd_next_bar || !reward_bar || !q_bar ||
      !qd_bar || !act_bar)
    return SHAC_ERR_INVALID_ARG;
  return run_adjoint(b, (cudaStream_t)stream, ws, 1, q, qd, act, reward_bar, nullptr, nullptr, q_next_bar, qd_next_bar,
                     q_bar, qd_bar, act_bar);
}

extern "C" shac_status shac_window_forward(shac_batch* b, void* stream, void* ws, int32_t h, const float* q0,
                                           const float* qd0, const float* act, float* q_traj, float* qd_traj,
                                           float* reward) {
  if (!b || !aligned_ws(b, ws) || h < 1 || h > b->h_max || !q0 || !qd0 || !act || !q_traj || !qd_traj || !reward)
    return SHAC_ERR_INVALID_ARG;
  return run_forward(b, (cudaStream_t)stream, ws, h, q0, qd0, act, q_traj + b->q_size, qd_traj + b->qd_size, reward,
                     q_traj, qd_traj, nullptr, true);
}

extern "C" shac_status shac_window_adjoint(shac_batch* b, void* stream, void* ws, int32_t h, const float* q_traj,
                                           const float* qd_traj, const float* act, const float* reward_bar,
                                           const float* q_traj_bar, const float* qd_traj_bar, float* q0_bar,
                                           float* qd0_bar, float* act_bar) {
  if (!b || !aligned_ws(b, ws) || h < 1 || h > b->h_max || !q_traj || !qd_traj || !act || !reward_bar || !q_traj_bar ||
      !qd_traj_bar || !q0_bar || !qd0_bar || !act_bar)
    return SHAC_ERR_INVALID_ARG;
  return run_adjoint(b, (cudaStream_t)stream, ws, h, q_traj, qd_traj, act, reward_bar, q_traj_bar, qd_traj_bar,
                     q_traj_bar + (size_t)h * b->q_size, qd_traj_bar + (size_t)h * b->qd_size, q0_bar, qd0_bar,
                     act_bar, nullptr, true);
}

extern "C" shac_status shac_window_forward_episodic(shac_batch* b, void* stream, void* ws, int32_t h,
                                                    const float* q0, const float* qd0, const float* act,
                                                    const float* q_reset, const float* qd_reset,
                                                    const float* term_height, const int32_t* max_episode_steps,
                                                    int32_t* episode_step, float* q_traj, float* qd_traj,
                                                    float* reward, uint8_t* done) {
  if (!b || !aligned_ws(b, ws) || h < 1 || h > b->h_max || !q0 || !qd0 || !act || !q_reset || !qd_reset ||
      !term_height || !max_episode_steps || !episode_step || !q_traj || !qd_traj || !reward || !done)
    return SHAC_ERR_INVALID_ARG;
  if (b->form != SHAC_FORM_BATCHED) return SHAC_ERR_UNSUPPORTED;
  Episodic ep;
  ep.q_reset = q_reset; ep.qd_reset = qd_reset; ep.term_height = term_height;
  ep.max_ep = max_episode_steps; ep.ep_step = episode_step; ep.done = done;
  return run_forward(b, (cudaStream_t)stream, ws, h, q0, qd0, act, q_traj + b->q_size, qd_traj + b->qd_size, reward,
                     q_traj, qd_traj, &ep, true);
}

extern "C" shac_status shac_window_adjoint_episodic(shac_batch* b, void* stream, void* ws, int32_t h,
                                                    const float* q_traj, const float* qd_traj, const float* act,
                                                    const uint8_t* done, const float* reward_bar,
                                                    const float* q_traj_bar, const float* qd_traj_bar,
                                                    float* q0_bar, float* qd0_bar, float* act_bar) {
  if (!b || !aligned_ws(b, ws) || h < 1 || h > b->h_max || !q_traj || !qd_traj || !act || !done || !reward_bar ||
      !q_traj_bar || !qd_traj_bar || !q0_bar || !qd0_bar || !act_bar)
    return SHAC_ERR_INVALID_ARG;
  if (b->form != SHAC_FORM_BATCHED) return SHAC_ERR_UNSUPPORTED;
  Episodic ep;
  ep.done_in = done;
  return run_adjoint(b, (cudaStream_t)stream, ws, h, q_traj, qd_traj, act, reward_bar, q_traj_bar, qd_traj_bar,
                     q_traj_bar + (size_t)h * b->q_size, qd_traj_bar + (size_t)h * b->qd_size, q0_bar, qd0_bar,
                     act_bar, &ep, true);
}

// ---------------------------------------------------------------------------
// Step adjoint with its scratch in a fixed device array of this library.
//
// Some callers cannot allocate device memory at the point where they call the
// simulator: code recorded into a CUDA graph under a capture mode that forbids
// allocation, runtimes that only hand out pre-registered buffers, or hosts
// whose device allocator is owned by another component.  They call
// shac_step_adjoint_static, which computes exactly what shac_step_adjoint
// computes but takes its scratch (work counter and substep records) from the
// array below instead of a caller workspace.  The array is STATIC_SCRATCH_BYTES
// (64 MiB) on every GPU that loads the library and stays resident until the
// process exits.
constexpr size_t STATIC_SCRATCH_BYTES = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int STATIC_MAX_DEVICES = 64;
static std::mutex g_static_mutex;
static void* g_static_addr[STATIC_MAX_DEVICES] = {};

// Device address of the array on device `dev`, which must be the current
// device: looked up once per device (on the first call made with that device
// current) and cached for the life of the process.  A device reset
// (cudaDeviceReset) reloads the module, possibly at another address, so the
// library must not be used across one.
static shac_status static_scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= STATIC_MAX_DEVICES) return SHAC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return SHAC_ERR_CUDA;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return SHAC_OK;
}

extern "C" shac_status shac_step_adjoint_static(shac_batch* b, void* stream, const float* q, const float* qd,
                                                const float* act, const float* q_next_bar, const float* qd_next_bar,
                                                const float* reward_bar, float* q_bar, float* qd_bar,
                                                float* act_bar) {
  if (!b || !q || !qd || !act || !q_next_bar || !qd_next_bar || !reward_bar || !q_bar || !qd_bar || !act_bar)
    return SHAC_ERR_INVALID_ARG;
  if (b->ws_step > STATIC_SCRATCH_BYTES) return SHAC_ERR_CAPACITY;
  // the array used is the current device's: it must be the GPU that holds the
  // batch's model tables and work items
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SHAC_ERR_CUDA;
  if (dev != b->device) return SHAC_ERR_INVALID_ARG;
  void* ws = nullptr;
  const shac_status st = static_scratch_address(dev, &ws);
  if (st != SHAC_OK) return st;
  return run_adjoint(b, (cudaStream_t)stream, ws, 1, q, qd, act, reward_bar, nullptr, nullptr, q_next_bar, qd_next_bar,
                     q_bar, qd_bar, act_bar);
}

extern "C" shac_status shac_get_status(shac_batch* b, void* stream, uint32_t* flags, int32_t clear) {
  if (!b || !flags) return SHAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned int v = 0;
  if (cudaMemcpyAsync(&v, b->d_flags, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SHAC_ERR_CUDA;
  *flags = v;
  if (clear && cudaMemsetAsync(b->d_flags, 0, sizeof(unsigned int), s) != cudaSuccess) return SHAC_ERR_CUDA;
  return (v & FLAG_NONFINITE) ? SHAC_ERR_NONFINITE : SHAC_OK;
}

extern "C" const char* shac_status_string(shac_status s) {
  switch (s) {
    case SHAC_OK: return "ok";
    case SHAC_ERR_INVALID_ARG: return "invalid argument";
    case SHAC_ERR_MODEL: return "malformed model";
    case SHAC_ERR_CUDA: return "CUDA runtime error";
    case SHAC_ERR_NONFINITE: return "non-finite state";
    case SHAC_ERR_CAPACITY: return "capacity exceeded";
    case SHAC_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

// -------------------------------------------------------------- autotune --
// Inputs and outputs of the autotuner's timed windows (h = min(h_max, 8)
// steps), carved from the caller's workspace after the batch's own part.
static const int AUTOTUNE_MAX_H = 8;
// A candidate shape replaces the best one only when its window is faster by
// more than this fraction (timing noise between equal shapes is ~1-3 %).
static const float AUTOTUNE_MARGIN = 0.03f;

static size_t autotune_parts(const shac_batch* b, size_t* parts) {
  const size_t h = (size_t)std::min(b->h_max, AUTOTUNE_MAX_H);
  const size_t nq = (size_t)b->q_size, nqd = (size_t)b->qd_size, na = (size_t)b->act_size, ne = (size_t)b->n_envs;
  const size_t p[12] = {nq, nqd, h * na, (h + 1) * nq, (h + 1) * nqd, h * ne, h * ne, (h + 1) * nq,
                        (h + 1) * nqd, nq, nqd, h * na};
  size_t total = 0;
  for (int k = 0; k < 12; ++k) {
    parts[k] = (p[k] + 63) / 64 * 64;   // 256-byte aligned pieces
    total += parts[k];
  }
  return total * sizeof(float);
}

extern "C" size_t shac_autotune_workspace_bytes(const shac_batch* b) {
  if (!b) return 0;
  size_t parts[12];
  return b->ws_total + autotune_parts(b, parts);
}

extern "C" shac_status shac_autotune(shac_batch* b, void* stream, void* ws, int32_t budget_ms, const float* q0_in,
                                     const float* qd0_in, const float* act_in) {
  if (!b || !aligned_ws(b, ws) || budget_ms <= 0) return SHAC_ERR_INVALID_ARG;
  if (b->form != SHAC_FORM_BATCHED || b->n_items == 0) return SHAC_OK;
  const auto t0 = std::chrono::steady_clock::now();
  auto out_of_time = [&]() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() > budget_ms;
  };
  cudaStream_t s = (cudaStream_t)stream;
  const int h = std::min(b->h_max, AUTOTUNE_MAX_H);
  const size_t nq = (size_t)b->q_size, nqd = (size_t)b->qd_size;
  size_t parts[12];
  const size_t buf_bytes = autotune_parts(b, parts);
  // the timed windows' buffers follow the batch's workspace (the launch shape
  // does not change its size)
  float* buf = reinterpret_cast<float*>(static_cast<char*>(ws) + b->ws_total);
  float* ptr[12];
  {
    size_t off = 0;
    for (int k = 0; k < 12; ++k) { ptr[k] = buf + off; off += parts[k]; }
  }
  float *q0 = ptr[0], *qd0 = ptr[1], *act = ptr[2], *qt = ptr[3], *qdt = ptr[4], *rew = ptr[5], *rbar = ptr[6];
  float *qtb = ptr[7], *qdtb = ptr[8], *q0b = ptr[9], *qd0b = ptr[10], *actb = ptr[11];
  // rest configuration: free joints at the origin with the identity quaternion (x, y, z, w: w = 1)
  std::vector<float> qh(nq, 0.f);
  for (int gi = 0; gi < (int)b->groups.size(); ++gi) {
    const Group& g = b->groups[gi];
    for (int i = 0; i < g.m->L; ++i)
      if (g.m->jtype[i] == J_FREE)
        for (int e = 0; e < g.N; ++e) qh[(size_t)b->io.g[gi].q_off + (size_t)(g.m->qs[i] + 6) * g.N + e] = 1.f;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  shac_status st = cuda_ok(cudaMemsetAsync(buf, 0, buf_bytes, s));
  if (st == SHAC_OK) st = cuda_ok(cudaMemcpyAsync(q0, qh.data(), nq * sizeof(float), cudaMemcpyHostToDevice, s));
  // the caller's window inputs replace the rest configuration where given
  if (st == SHAC_OK && q0_in)
    st = cuda_ok(cudaMemcpyAsync(q0, q0_in, nq * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (st == SHAC_OK && qd0_in)
    st = cuda_ok(cudaMemcpyAsync(qd0, qd0_in, nqd * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (st == SHAC_OK && act_in)
    st = cuda_ok(cudaMemcpyAsync(act, act_in, (size_t)h * b->act_size * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (st == SHAC_OK) st = cuda_ok(cudaStreamSynchronize(s));   // qh is a host temporary
  if (st == SHAC_OK) st = cuda_ok(cudaEventCreate(&e0));
  if (st == SHAC_OK) st = cuda_ok(cudaEventCreate(&e1));
  auto window = [&]() -> shac_status {
    shac_status r = run_forward(b, s, ws, h, q0, qd0, act, qt + nq, qdt + nqd, rew, qt, qdt, nullptr, true);
    if (r != SHAC_OK) return r;
    return run_adjoint(b, s, ws, h, qt, qdt, act, rbar, qtb, qdtb, qtb + (size_t)h * nq, qdtb + (size_t)h * nqd,
                       q0b, qd0b, actb, nullptr, true);
  };
  // ms per window of the current shape: median of three after one warm-up
  // (infinite if the shape does not launch)
  auto measure = [&](float* ms) -> shac_status {
    *ms = INFINITY;
    shac_status r = window();
    if (r == SHAC_ERR_CAPACITY) return SHAC_OK;
    if (r != SHAC_OK) return r;
    float t[3];
    for (int rep = 0; rep < 3; ++rep) {
      if (cudaEventRecord(e0, s) != cudaSuccess) return SHAC_ERR_CUDA;
      if ((r = window()) != SHAC_OK) return r;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return SHAC_ERR_CUDA;
      if (cudaEventElapsedTime(&t[rep], e0, e1) != cudaSuccess) return SHAC_ERR_CUDA;
    }
    std::sort(t, t + 3);
    *ms = t[1];
    return SHAC_OK;
  };
  auto better = [](float t, float best) { return t < best * (1.f - AUTOTUNE_MARGIN); };
  const int n_groups = (int)b->groups.size();
  std::vector<int> lanes0(n_groups), best_lanes(n_groups);
  for (int gi = 0; gi < n_groups; ++gi) lanes0[gi] = best_lanes[gi] = b->groups[gi].lanes;
  const int warps0 = b->warps_per_cta;
  int best_warps = warps0;
  float best = INFINITY;
  if (st == SHAC_OK) st = measure(&best);
  static const int kLanes[] = {1, 2, 4, 8, 16, 32};
  static const int kWarps[] = {1, 2, 4, 8};
  // a specialised batch keeps the team size its kernels were compiled for
  // (other team sizes would run the generic kernels, which rank shapes
  // differently) and searches the warps per CTA with its own kernels
  const bool specialised = b->spec.key != 0 && b->spec_lanes == b->groups[0].lanes;
  for (int gi = 0; gi < n_groups && st == SHAC_OK && !out_of_time() && !specialised; ++gi) {
    if (b->groups[gi].N == 0) continue;
    for (int l : kLanes) {
      if (st != SHAC_OK || out_of_time()) break;
      if (l == best_lanes[gi]) continue;
      for (int gj = 0; gj < n_groups; ++gj) b->groups[gj].lanes = best_lanes[gj];
      b->groups[gi].lanes = l;
      b->warps_per_cta = best_warps;
      if ((st = build_items(b)) != SHAC_OK) break;
      float t;
      if ((st = measure(&t)) == SHAC_OK && better(t, best)) { best = t; best_lanes[gi] = l; }
    }
  }
  for (int w : kWarps) {
    if (st != SHAC_OK || out_of_time()) break;
    if (w == best_warps) continue;
    for (int gj = 0; gj < n_groups; ++gj) b->groups[gj].lanes = best_lanes[gj];
    b->warps_per_cta = w;
    if ((st = build_items(b)) != SHAC_OK) break;
    float t;
    if ((st = measure(&t)) == SHAC_OK && better(t, best)) { best = t; best_warps = w; }
  }
  // keep the best shape (the starting one after an error)
  const bool ok = st == SHAC_OK;
  for (int gj = 0; gj < n_groups; ++gj) b->groups[gj].lanes = ok ? best_lanes[gj] : lanes0[gj];
  b->warps_per_cta = ok ? best_warps : warps0;
  const shac_status st_items = build_items(b);
  cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != SHAC_OK) return st;
  return st_items;
}
