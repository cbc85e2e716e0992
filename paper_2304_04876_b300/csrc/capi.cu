// C ABI entry points of libgdsw (declared in include/gdsw.h).
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>
#include <thread>
#include <atomic>

#include "internal.h"

struct gdsw_ctx {
  gdsw::Ctx c;
  // kept for gdsw_refactor: the symbolic plan, the CSR pattern and the null space
  gdsw::Plan plan;
  std::vector<int> rowptr, colind;
  std::vector<double> Z;
  int32_t nn = 0;
};

namespace gdsw {

namespace {
thread_local char g_err[512] = "";

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void release(Ctx* c) {
  if (c->bgraph_exec) cudaGraphExecDestroy(c->bgraph_exec);
  if (c->bgraph) cudaGraphDestroy(c->bgraph);
  if (c->sgraph_exec) cudaGraphExecDestroy(c->sgraph_exec);
  if (c->sgraph) cudaGraphDestroy(c->sgraph);
  if (c->bks_host) cudaFreeHost(c->bks_host);
  if (c->bgraph_stream) cudaStreamDestroy(c->bgraph_stream);
  if (c->gm_exec) cudaGraphExecDestroy(c->gm_exec);
  if (c->gm_graph) cudaGraphDestroy(c->gm_graph);
  if (c->pcg_exec) cudaGraphExecDestroy(c->pcg_exec);
  if (c->pcg_graph) cudaGraphDestroy(c->pcg_graph);
  if (c->graph_stream) cudaStreamDestroy(c->graph_stream);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_x) cudaEventDestroy(c->ev_x);
  if (c->ev_xdone) cudaEventDestroy(c->ev_xdone);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->ks_host) cudaFreeHost(c->ks_host);
  if (c->hpin) cudaFreeHost(c->hpin);
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
}

bool valid_options(const gdsw_options* o) {
  return o->local_solver >= 0 && o->local_solver <= 2 && o->trsv >= 0 && o->trsv <= 1 &&
         o->sweeps_factor >= 0 && o->sweeps_trsv >= 0 && o->overlap >= 0 && o->precision >= 0 &&
         o->precision <= 2 && o->krylov >= 0 && o->krylov <= 1 && o->restart >= 1 &&
         o->maxit >= 1 && o->coarse >= 0 && o->coarse <= 2 && o->tol > 0.0 && o->wait_budget_cycles >= 0 &&
         o->fill_level >= 0 && (o->fill_level == 0 || o->local_solver != GDSW_LOCAL_EXACT) &&
         (o->autotune == 0 || o->autotune == 1) && (o->gmres_orth >= 0 && o->gmres_orth <= 2);
}
}  // namespace

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

gdsw_status apply_configure(Ctx* c);

// One solve on any handle; for a batch, info summarises every member (largest
// iteration count and residual, converged only if all converged).
gdsw_status solve_any(Ctx* c, const double* b, double* x, gdsw_solve_info* info, cudaStream_t s) {
  if (c->nprob > 1) {
    std::vector<gdsw_solve_info> all(c->nprob);
    gdsw_status st = solve_batch(c, b, x, all.data(), s);
    if (info) {
      *info = gdsw_solve_info{0, 1, 0.0, 0.0};
      for (const auto& a : all) {
        info->iters = std::max(info->iters, a.iters);
        info->converged = info->converged && a.converged;
        info->true_relres = std::max(info->true_relres, a.true_relres);
        info->seconds = a.seconds;
      }
    }
    return st;
  }
  return c->opt.krylov == GDSW_KRYLOV_GMRES ? solve_gmres(c, b, x, info, s) : solve_pcg(c, b, x, info, s);
}

}  // namespace gdsw

using namespace gdsw;

extern "C" {

void gdsw_default_options(gdsw_options* o) {
  if (!o) return;
  o->local_solver = GDSW_LOCAL_IC0;
  o->trsv = GDSW_TRSV_LEVELSCHED;
  o->sweeps_factor = 3;
  o->sweeps_trsv = 5;
  o->overlap = 1;
  o->precision = GDSW_PREC_FP64;
  o->krylov = GDSW_KRYLOV_PCG;
  o->restart = 30;
  o->maxit = 2000;
  o->coarse = GDSW_COARSE_GDSW;
  o->fill_level = 0;
  o->autotune = 1;
  o->gmres_orth = GDSW_GMRES_ORTH_CGS2;
  o->flexible = -1;
  o->tol = 1e-8;
  o->wait_budget_cycles = 0;
}

const char* gdsw_status_string(gdsw_status s) {
  switch (s) {
    case GDSW_OK: return "ok";
    case GDSW_ERR_INVALID_ARG: return "invalid argument";
    case GDSW_ERR_OUT_OF_MEMORY: return "out of device memory";
    case GDSW_ERR_BREAKDOWN: return "factorization breakdown";
    case GDSW_ERR_NOT_CONVERGED: return "not converged";
    case GDSW_ERR_TIMEOUT: return "device wait timed out";
    case GDSW_ERR_CUDA: return "CUDA error";
    case GDSW_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* gdsw_last_error(void) { return g_err; }

}  // extern "C"

namespace {

// Numeric setup, apply/SpMV configuration and Krylov workspace for a plan
// (one problem, or the merged plan of a batch); the handle on success.
gdsw_status setup_from_plan(const Plan& P, const gdsw_csr* A, const double* Z, int32_t nn,
                            const gdsw_options& o, cudaStream_t s, double t0, double t_sym,
                            gdsw_handle* out, std::shared_ptr<const MfPlan> mf_plan = nullptr) {
  gdsw_ctx* h = new (std::nothrow) gdsw_ctx();
  if (!h) { set_error("host allocation failed"); return GDSW_ERR_OUT_OF_MEMORY; }
  Ctx* c = &h->c;
  c->mf_plan_host = std::move(mf_plan);
  cudaGetDevice(&c->device);
  c->opt = o;
  c->n = P.n;
  c->nnz = P.nnz;
  c->nsub = P.nsub;
  c->ncomp = P.ncomp;
  c->dpn = P.dpn;
  c->max_m = P.max_m;
  c->sum_m = P.sum_m;
  c->nprob = P.nprob;
  c->fp32 = o.precision == GDSW_PREC_FP32 || o.precision == GDSW_PREC_FP16;
  c->fp16 = o.precision == GDSW_PREC_FP16;
  c->flexible = o.flexible < 0 ? c->fp32 : (o.flexible != 0);
  c->wait_cycles = o.wait_budget_cycles > 0 ? o.wait_budget_cycles : kDefaultWaitCycles;
  c->stats.setup_phase_seconds[0] = t_sym;
  gdsw_status st = numeric_setup(c, P, A, Z, nn, s);
  if (st == GDSW_OK) st = c->fp32 ? dalloc(c, reinterpret_cast<float**>(&c->zloc), P.sum_m)
                                  : dalloc(c, reinterpret_cast<double**>(&c->zloc), P.sum_m);
  if (st == GDSW_OK) st = apply_configure(c);
  if (st == GDSW_OK) st = spmv_configure(c, A->rowptr, A->colind, A->val);
  const double t1 = now_s();
  if (st == GDSW_OK) st = krylov_init(c, s);
  if (st == GDSW_OK && P.nprob > 1) {
    // problem of each subdomain (from its first unknown; subdomains are
    // concatenated problem by problem) and of each Phi block
    std::vector<int> sub_prob(P.nsub, 0), blk_prob;
    for (int q = 0; q < P.nsub; ++q) {
      if (P.om_ptr[q + 1] > P.om_ptr[q]) {
        const int dof = P.om_dofs[P.om_ptr[q]];
        sub_prob[q] = static_cast<int>(std::upper_bound(P.prob_dof_ptr.begin(), P.prob_dof_ptr.end(), dof) -
                                       P.prob_dof_ptr.begin()) - 1;
      } else {
        sub_prob[q] = q > 0 ? sub_prob[q - 1] : 0;
      }
    }
    blk_prob = sub_prob;
    blk_prob.insert(blk_prob.end(), P.comp_prob.begin(), P.comp_prob.end());
    blk_prob.resize(std::max(c->nblk, P.nsub + P.ncomp), 0);
    st = batch_init(c, P.prob_dof_ptr, sub_prob, blk_prob, s);
  }
  if (st == GDSW_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_error("setup: %s", cudaGetErrorString(e)); st = GDSW_ERR_CUDA; }
  }
  if (st != GDSW_OK) {
    release(c);
    delete h;
    return st;
  }
  c->stats.setup_phase_seconds[7] = now_s() - t1;
  gdsw_stats& S = c->stats;
  S.n = P.n;
  S.nnz = P.nnz;
  S.n_sub = P.nsub;
  S.n0 = c->n0;
  S.n_comp = P.ncomp;
  S.sum_omega = P.sum_m;
  S.max_omega = P.max_m;
  S.nnz_L = P.L.nnz;
  S.nnz_U = P.U.nnz;
  S.ell_L = P.L.slots;
  S.ell_U = P.U.slots;
  S.n_levels_L = static_cast<int64_t>(P.L.lev_nr.size());
  S.n_levels_U = static_cast<int64_t>(P.U.lev_nr.size());
  S.max_levels = c->max_levels;
  S.n_blocks = c->nblk;
  S.device_bytes = static_cast<int64_t>(c->bytes);
  S.n_problems = P.nprob;
  S.local_stages = c->node_stages > 0 ? c->node_stages : c->step_depth > 0 ? c->step_depth : c->rec_stages;
  S.local_threads = c->jac_mode > 0 ? c->jac_threads : c->node_stages > 0 ? c->node_threads
                  : c->step_depth > 0 ? kStepRows : c->rec_stages > 0 ? c->rec_consumers : c->tri_threads;
  S.local_kernel = c->mf ? 1 : o.local_solver == GDSW_LOCAL_EXACT ? 0 : c->jac_mode > 0 ? 5
                 : c->node_stages > 0 ? 7 : c->step_depth > 0 ? 6 : c->rec_stages > 0 ? (c->rec_sf ? 4 : 3) : 2;
  S.pcg_persistent_grid = c->persist_grid;
  S.phi_beside_local = c->prolong;
  S.phiT_wide = c->phiT_wide ? 1 : 0;
  S.setup_seconds = now_s() - t0;
  *out = h;
  return GDSW_OK;
}

// The handle remembers what gdsw_refactor needs to rerun the numeric phase.
void keep_for_refactor(gdsw_handle h, Plan&& P, std::vector<int>&& rp, std::vector<int>&& ci, const double* Z,
                       int32_t nn) {
  h->plan = std::move(P);
  h->rowptr = std::move(rp);
  h->colind = std::move(ci);
  if (Z && nn > 0) h->Z.assign(Z, Z + int64_t(h->plan.n) * nn);
  h->nn = Z ? nn : 0;
}

bool prepare_options(const gdsw_options* opt, gdsw_options* o) {
  if (opt) *o = *opt; else gdsw_default_options(o);
  if (!valid_options(o)) { set_error("invalid options"); return false; }
  return true;
}

// A host view of a CSR matrix: the caller's arrays for GDSW_MEM_HOST, host
// copies of device arrays for GDSW_MEM_DEVICE.
struct HostCsr {
  gdsw_csr view{};
  std::vector<int32_t> rp, ci;
  std::vector<double> va;
};

gdsw_status host_csr(const gdsw_csr* A, HostCsr* H) {
  if (!A) { set_error("null matrix"); return GDSW_ERR_INVALID_ARG; }
  if (A->mem == GDSW_MEM_HOST) { H->view = *A; return GDSW_OK; }
  if (A->mem != GDSW_MEM_DEVICE) { set_error("gdsw_csr.mem = %d is neither host nor device", A->mem); return GDSW_ERR_INVALID_ARG; }
  if (A->n <= 0 || !A->rowptr || !A->colind || !A->val) { set_error("null or empty device CSR"); return GDSW_ERR_INVALID_ARG; }
  H->rp.resize(size_t(A->n) + 1);
  GDSW_CK(cudaMemcpy(H->rp.data(), A->rowptr, H->rp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
  const int64_t nnz = H->rp[A->n];
  if (H->rp[0] != 0 || nnz < A->n || nnz >= (int64_t(1) << 31)) { set_error("device rowptr is not a CSR row pointer"); return GDSW_ERR_INVALID_ARG; }
  H->ci.resize(nnz);
  H->va.resize(nnz);
  GDSW_CK(cudaMemcpy(H->ci.data(), A->colind, size_t(nnz) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  GDSW_CK(cudaMemcpy(H->va.data(), A->val, size_t(nnz) * sizeof(double), cudaMemcpyDeviceToHost));
  H->view = gdsw_csr{A->n, H->rp.data(), H->ci.data(), H->va.data(), GDSW_MEM_HOST};
  return GDSW_OK;
}

}  // namespace

extern "C" {

gdsw_status gdsw_setup(const gdsw_csr* A, const gdsw_partition* part, const double* Z, int32_t nn,
                       const gdsw_options* opt, void* stream, gdsw_handle* out) {
  if (!out) { set_error("null output handle"); return GDSW_ERR_INVALID_ARG; }
  *out = nullptr;
  gdsw_options o;
  if (!prepare_options(opt, &o)) return GDSW_ERR_INVALID_ARG;
  if (nn < 0 || (nn > 0 && !Z)) { set_error("null space: nn=%d with Z=%p", nn, (const void*)Z); return GDSW_ERR_INVALID_ARG; }
  const double t0 = now_s();
  HostCsr H;
  GDSW_TRY(host_csr(A, &H));
  A = &H.view;
  Plan P;
  gdsw_status st = build_plan(A, part, &o, o.local_solver != GDSW_LOCAL_EXACT, &P);
  if (st != GDSW_OK) return st;
  st = setup_from_plan(P, A, Z, nn, o, static_cast<cudaStream_t>(stream), t0, now_s() - t0, out);
  if (st == GDSW_OK)
    keep_for_refactor(*out, std::move(P), std::vector<int>(A->rowptr, A->rowptr + A->n + 1),
                      std::vector<int>(A->colind, A->colind + A->rowptr[A->n]), Z, nn);
  return st;
}

gdsw_status gdsw_bytes_required(const gdsw_csr* A, const gdsw_partition* part, const double* Z, int32_t nn,
                                const gdsw_options* opt, int64_t* resident, int64_t* setup_scratch) {
  gdsw_options o;
  if (!prepare_options(opt, &o)) return GDSW_ERR_INVALID_ARG;
  if (nn < 0 || (nn > 0 && !Z)) { set_error("null space: nn=%d with Z=%p", nn, (const void*)Z); return GDSW_ERR_INVALID_ARG; }
  HostCsr H;
  GDSW_TRY(host_csr(A, &H));
  A = &H.view;
  Plan P;
  gdsw_status st = build_plan(A, part, &o, o.local_solver != GDSW_LOCAL_EXACT, &P);
  if (st != GDSW_OK) return st;
  int64_t r = 0, sc = 0;
  st = estimate_footprint(P, A, o, Z ? nn : 0, &r, &sc);
  if (st != GDSW_OK) return st;
  if (resident) *resident = r;
  if (setup_scratch) *setup_scratch = sc;
  return GDSW_OK;
}

gdsw_status gdsw_mf_plan_export(const gdsw_csr* A, const gdsw_partition* part, const gdsw_options* opt,
                                int32_t subdomain, int32_t* m, int32_t* nsn, int64_t* nb_total,
                                int32_t* nd_dof, int32_t* sn_ptr, int32_t* parent, int64_t* b_ptr,
                                int32_t* b_pos) {
  gdsw_options o;
  if (!prepare_options(opt, &o)) return GDSW_ERR_INVALID_ARG;
  if (!m || !nsn || !nb_total) { set_error("null size output"); return GDSW_ERR_INVALID_ARG; }
  HostCsr H;
  GDSW_TRY(host_csr(A, &H));
  A = &H.view;
  Plan P;
  gdsw_status st = build_plan(A, part, &o, false, &P);
  if (st != GDSW_OK) return st;
  if (subdomain < 0 || subdomain >= P.nsub) {
    set_error("subdomain %d outside [0, %d)", subdomain, P.nsub);
    return GDSW_ERR_INVALID_ARG;
  }
  MfPlan M;
  st = build_mf_plan(P, mf_leaf_size(), mf_buf_bytes(4) / 4, &M);
  if (st != GDSW_OK) return st;
  const int q = subdomain, base = P.om_ptr[q];
  const int s0 = M.sub_sn[q], s1 = M.sub_sn[q + 1];
  *m = P.om_ptr[q + 1] - base;
  *nsn = s1 - s0;
  int64_t nb = 0;
  for (int S = s0; S < s1; ++S) nb += M.sn[S].nb;
  *nb_total = nb;
  if (nd_dof)
    for (int p = 0; p < *m; ++p) nd_dof[p] = M.nd_dof[base + p];
  if (sn_ptr) {
    for (int S = s0; S < s1; ++S) sn_ptr[S - s0] = M.sn[S].pos0;
    sn_ptr[s1 - s0] = *m;
  }
  if (parent) {
    for (int S = s0; S < s1; ++S) parent[S - s0] = -1;
    for (int S = s0; S < s1; ++S)
      for (int t = M.ch_ptr[S]; t < M.ch_ptr[S + 1]; ++t) parent[M.ch_list[t] - s0] = S - s0;
  }
  if (b_ptr || b_pos) {
    int64_t k = 0;
    for (int S = s0; S < s1; ++S) {
      if (b_ptr) b_ptr[S - s0] = k;
      for (int r = 0; r < M.sn[S].nb; ++r, ++k)
        if (b_pos) b_pos[k] = M.bidx[M.sn[S].brow + r];
    }
    if (b_ptr) b_ptr[s1 - s0] = k;
  }
  return GDSW_OK;
}

gdsw_status gdsw_refactor(gdsw_handle h, const double* val, void* stream) {
  if (!h || !val) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  const double t0 = now_s();
  gdsw_csr A{h->plan.n, h->rowptr.data(), h->colind.data(), val};
  gdsw_handle fresh = nullptr;
  gdsw_status st = setup_from_plan(h->plan, &A, h->Z.empty() ? nullptr : h->Z.data(), h->nn, h->c.opt,
                                   static_cast<cudaStream_t>(stream), t0, 0.0, &fresh, h->c.mf_plan_host);
  if (st != GDSW_OK) return st;           // the handle keeps its previous factors
  std::swap(h->c, fresh->c);
  release(&fresh->c);
  delete fresh;
  return GDSW_OK;
}

gdsw_status gdsw_setup_batch(int32_t count, const gdsw_csr* A, const gdsw_partition* parts,
                             const double* const* Z, const int32_t* nn, const gdsw_options* opt,
                             void* stream, gdsw_handle* out) {
  if (!out) { set_error("null output handle"); return GDSW_ERR_INVALID_ARG; }
  *out = nullptr;
  if (count < 1 || !A || !parts) { set_error("batch needs count >= 1 matrices and partitions"); return GDSW_ERR_INVALID_ARG; }
  gdsw_options o;
  if (!prepare_options(opt, &o)) return GDSW_ERR_INVALID_ARG;
  if (o.krylov == GDSW_KRYLOV_GMRES && o.gmres_orth == GDSW_GMRES_ORTH_DCGS2) {
    set_error("batched GMRES uses CGS2 or the single-reduce form");
    return GDSW_ERR_UNSUPPORTED;
  }
  const double t0 = now_s();
  std::vector<HostCsr> hosts(count);
  for (int p = 0; p < count; ++p) GDSW_TRY(host_csr(&A[p], &hosts[p]));
  std::vector<gdsw_csr> views(count);
  for (int p = 0; p < count; ++p) views[p] = hosts[p].view;
  A = views.data();
  std::vector<Plan> plans(count);
  int nnmax = 1;
  int64_t n = 0, nnz = 0;
  for (int p = 0; p < count; ++p) {
    const int np_ = nn ? nn[p] : 0;
    if (np_ < 0 || (np_ > 0 && (!Z || !Z[p]))) { set_error("null space of member %d", p); return GDSW_ERR_INVALID_ARG; }
    nnmax = std::max(nnmax, np_);
    n += A[p].n;
    nnz += A[p].rowptr[A[p].n];
  }
  {
    // the members' symbolic phases are independent: host threads take them in
    // turn; a member that fails is built again on this thread, which sets the
    // error message
    std::vector<gdsw_status> sts(count, GDSW_OK);
    std::atomic<int> next{0};
    const bool levels = o.local_solver != GDSW_LOCAL_EXACT;
    auto work = [&]() {
      for (int p = next++; p < count; p = next++) sts[p] = build_plan(&A[p], &parts[p], &o, levels, &plans[p]);
    };
    const int nth = std::max(1, std::min<int>(count, static_cast<int>(std::thread::hardware_concurrency())));
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t) pool.emplace_back(work);
    work();
    for (auto& th : pool) th.join();
    for (int p = 0; p < count; ++p)
      if (sts[p] != GDSW_OK) return build_plan(&A[p], &parts[p], &o, levels, &plans[p]);
  }
  if (n >= (int64_t(1) << 31) || nnz >= (int64_t(1) << 31)) { set_error("batch too large"); return GDSW_ERR_UNSUPPORTED; }
  // block-diagonal union: CSR and null space (missing columns stay zero and are
  // dropped by the orthonormalisation)
  std::vector<int> rp(n + 1, 0), ci;
  std::vector<double> va;
  ci.reserve(nnz);
  va.reserve(nnz);
  std::vector<double> Zm(size_t(n) * nnmax, 0.0);
  int64_t off = 0;
  for (int p = 0; p < count; ++p) {
    const gdsw_csr& a = A[p];
    for (int i = 0; i < a.n; ++i) {
      for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
        ci.push_back(static_cast<int>(a.colind[e] + off));
        va.push_back(a.val[e]);
      }
      rp[off + i + 1] = static_cast<int>(ci.size());
    }
    const int np_ = nn ? nn[p] : 0;
    for (int col = 0; col < nnmax; ++col)
      for (int i = 0; i < a.n; ++i)
        Zm[size_t(col) * n + off + i] = np_ == 0 ? (col == 0 ? 1.0 : 0.0)
                                                 : (col < np_ ? Z[p][size_t(col) * a.n + i] : 0.0);
    off += a.n;
  }
  Plan M;
  gdsw_status st = merge_plans(plans, &M);
  if (st != GDSW_OK) return st;
  gdsw_csr merged{static_cast<int32_t>(n), rp.data(), ci.data(), va.data()};
  st = setup_from_plan(M, &merged, Zm.data(), nnmax, o, static_cast<cudaStream_t>(stream), t0, now_s() - t0, out);
  if (st == GDSW_OK) keep_for_refactor(*out, std::move(M), std::move(rp), std::move(ci), Zm.data(), nnmax);
  return st;
}

gdsw_status gdsw_get_stats(gdsw_handle h, gdsw_stats* st) {
  if (!h || !st) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  *st = h->c.stats;
  return GDSW_OK;
}

gdsw_status gdsw_apply(gdsw_handle h, const double* r, double* z, void* stream) {
  if (!h || !r || !z) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  return apply_enqueue(&h->c, r, z, static_cast<cudaStream_t>(stream), false);
}

gdsw_status gdsw_apply_timed(gdsw_handle h, const double* r, double* z, void* stream,
                             double* phase_ms) {
  if (!h || !r || !z || !phase_ms) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  return apply_timed(&h->c, r, z, static_cast<cudaStream_t>(stream), phase_ms);
}

gdsw_status gdsw_batch_start(gdsw_handle h, int32_t member, const double* b, void* stream) {
  if (!h || !b) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  Ctx* c = &h->c;
  if (c->nprob < 2 || c->bks == nullptr) { set_error("gdsw_batch_start needs a batched handle"); return GDSW_ERR_INVALID_ARG; }
  if (c->opt.krylov != GDSW_KRYLOV_PCG) { set_error("continuous batching runs PCG"); return GDSW_ERR_UNSUPPORTED; }
  if (member < 0 || member >= c->nprob) { set_error("member %d out of range [0, %d)", member, c->nprob); return GDSW_ERR_INVALID_ARG; }
  return batch_start(c, member, b, static_cast<cudaStream_t>(stream));
}

gdsw_status gdsw_batch_iterate(gdsw_handle h, int32_t iterations, void* stream) {
  if (!h || iterations < 0) { set_error("null handle or negative iteration count"); return GDSW_ERR_INVALID_ARG; }
  Ctx* c = &h->c;
  if (c->nprob < 2 || c->bks == nullptr) { set_error("gdsw_batch_iterate needs a batched handle"); return GDSW_ERR_INVALID_ARG; }
  if (c->opt.krylov != GDSW_KRYLOV_PCG) { set_error("continuous batching runs PCG"); return GDSW_ERR_UNSUPPORTED; }
  return batch_iterate(c, iterations, static_cast<cudaStream_t>(stream));
}

gdsw_status gdsw_batch_status(gdsw_handle h, int32_t* done, int32_t* iters, double* relres, void* stream) {
  if (!h) { set_error("null handle"); return GDSW_ERR_INVALID_ARG; }
  Ctx* c = &h->c;
  if (c->nprob < 2 || c->bks == nullptr) { set_error("gdsw_batch_status needs a batched handle"); return GDSW_ERR_INVALID_ARG; }
  return batch_status(c, done, iters, relres, static_cast<cudaStream_t>(stream));
}

gdsw_status gdsw_batch_finish(gdsw_handle h, int32_t member, double* x, gdsw_solve_info* info,
                              int32_t* continued, void* stream) {
  if (!h) { set_error("null handle"); return GDSW_ERR_INVALID_ARG; }
  Ctx* c = &h->c;
  if (c->nprob < 2 || c->bks == nullptr) { set_error("gdsw_batch_finish needs a batched handle"); return GDSW_ERR_INVALID_ARG; }
  if (member < 0 || member >= c->nprob) { set_error("member %d out of range [0, %d)", member, c->nprob); return GDSW_ERR_INVALID_ARG; }
  return batch_finish(c, member, x, info, continued, static_cast<cudaStream_t>(stream));
}

gdsw_status gdsw_pcg_iteration_timed(gdsw_handle h, const double* b, void* stream, double* kernel_ms) {
  if (!h || !b || !kernel_ms) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  return pcg_iteration_timed(&h->c, b, static_cast<cudaStream_t>(stream), kernel_ms);
}

gdsw_status gdsw_spmv(gdsw_handle h, const double* x, double* y, void* stream) {
  if (!h || !x || !y) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  return spmv_enqueue(&h->c, x, y, static_cast<cudaStream_t>(stream));
}

gdsw_status gdsw_solve(gdsw_handle h, const double* b, double* x, gdsw_solve_info* info,
                       void* stream) {
  if (!h || !b || !x) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  return solve_any(&h->c, b, x, info, static_cast<cudaStream_t>(stream));
}

gdsw_status gdsw_solve_batch(gdsw_handle h, const double* b, double* x, gdsw_solve_info* info,
                             void* stream) {
  if (!h || !b || !x) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  Ctx* c = &h->c;
  if (c->nprob == 1) return solve_any(c, b, x, info, static_cast<cudaStream_t>(stream));
  return solve_batch(c, b, x, info, static_cast<cudaStream_t>(stream));
}

gdsw_status gdsw_solve_host(gdsw_handle h, const double* b_host, double* x_host,
                            gdsw_solve_info* info, void* stream) {
  if (!h || !b_host || !x_host) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  Ctx* c = &h->c;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double t0 = now_s();
  const size_t bytes = sizeof(double) * c->n;
  // b and x0 travel into two workspace vectors that the solve copies from before
  // it first writes them (q is first written by the initial SpMV, p after the
  // initial residual)
  GDSW_CK(cudaMemcpyAsync(c->q, b_host, bytes, cudaMemcpyHostToDevice, s));
  GDSW_CK(cudaMemcpyAsync(c->p, x_host, bytes, cudaMemcpyHostToDevice, s));
  double* bd = c->q;
  double* xd = c->p;
  gdsw_status st = solve_any(c, bd, xd, info, s);
  if (st != GDSW_OK && st != GDSW_ERR_NOT_CONVERGED) return st;
  GDSW_CK(cudaMemcpyAsync(x_host, c->x, bytes, cudaMemcpyDeviceToHost, s));
  GDSW_CK(cudaStreamSynchronize(s));
  if (info) info->seconds = now_s() - t0;
  return st;
}

gdsw_status gdsw_solve_host_zero_guess(gdsw_handle h, const double* b_host, double* x_host,
                                       gdsw_solve_info* info, void* stream) {
  if (!h || !b_host || !x_host) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  Ctx* c = &h->c;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double t0 = now_s();
  const size_t bytes = sizeof(double) * c->n;
  // as gdsw_solve_host, with the initial guess set to zero on the device
  GDSW_CK(cudaMemcpyAsync(c->q, b_host, bytes, cudaMemcpyHostToDevice, s));
  GDSW_CK(cudaMemsetAsync(c->p, 0, bytes, s));
  gdsw_status st = solve_any(c, c->q, c->p, info, s);
  if (st != GDSW_OK && st != GDSW_ERR_NOT_CONVERGED) return st;
  GDSW_CK(cudaMemcpyAsync(x_host, c->x, bytes, cudaMemcpyDeviceToHost, s));
  GDSW_CK(cudaStreamSynchronize(s));
  if (info) info->seconds = now_s() - t0;
  return st;
}

gdsw_status gdsw_destroy(gdsw_handle h) {
  if (!h) return GDSW_OK;
  release(&h->c);
  delete h;
  return GDSW_OK;
}

}  // extern "C"
