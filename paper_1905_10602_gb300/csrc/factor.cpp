// IFMM factorization (Algorithm 1 with the colors of Algorithm 3).
//
// The host walks the symbolic structure (which blocks exist, their shapes, who
// is eliminated) and emits, per color, batches of descriptors for the dense
// device kernels; every arithmetic step runs on the GPU.  Per color:
//   phase A  for every node i of the color (independent for sigma >= 3):
//            Pi_i = [[P2P_ii, L2P_i], [P2M_i, 0]] -> Pi_i^{-1} (Gauss-Jordan),
//            Schur complement of the clique: F = -L Pi^{-1} U over the
//            neighbours' current rows/columns, added in place to near blocks;
//            far fill-ins (pairs of N_i in each other's interaction list) kept;
//            then every live neighbour that received far fill-ins gets new
//            orthonormal bases from weighted SVDs (recompression at eps).
//   (sync)   singular values come back to the host, which picks the ranks.
//   phase B  M2L / M2M / L2L blocks touching a re-based node are re-expressed,
//            M <- T'_a M T_b: the interaction-list updates that the paper
//            serializes for sigma = 3 (Sec. 3.3) become one deterministic pass.
//   phase C  fill-in coefficients in the new bases are added to M2L.
// Block state between two nodes at distance <= 1 lives in three "stage"
// buffers (both live / one eliminated / both eliminated), so the blocks the
// solve needs stay untouched once a stage ends.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <exception>
#include <functional>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <unordered_map>

#include "fact.h"
#include "host_pool.h"
#include "ifmm_kernels.h"
#include "mlp.h"

namespace ifmm {

// logical block op(src): rows x cols
struct Blk {
  const double* p;
  int ld, rows, cols, trans;
};

// host threads for a loop over n independent items (1 below 64 items): at most
// half the host's hardware threads and 8, unless IFMM_HOST_THREADS (read once
// per process) sets another maximum (below the hardware thread count)
static int host_threads(int n) {
  static const int hw = [] {
    const long h = std::max(2u, std::thread::hardware_concurrency());
    const char* e = getenv("IFMM_HOST_THREADS");
    const long want = e ? atol(e) : std::min(8L, h / 2);
    return (int)std::max(1L, std::min(want, h - 1));
  }();
  const int cap = host_thread_cap();
  const int lim = cap > 0 ? std::min(hw, cap) : hw;
  return n < 64 ? 1 : std::min(lim, n / 32);
}

static inline int64_t key3(int a, int b, int c) { return ((int64_t)a << 40) | ((int64_t)b << 20) | (int64_t)c; }

struct Work {
  int kappa = 0, nn = 0;
  const LevelLists* LL = nullptr;
  std::vector<int> n, r, capr;
  std::vector<int> elim;
  std::vector<int> slot_ptr;
  std::vector<double*> nb[3];
  std::vector<double*> far;  // indexed by position in the IL CSR
  std::vector<double*> P2M, L2P, M2M, L2L;
  std::vector<int> choff;  // offset of this node's y inside its parent's x
  std::vector<int> il_T;   // il_T[e] = position of (b, a) for the IL entry e = (a, b)
  std::vector<int> il_row; // il_row[e] = a for the IL entry e = (a, b)
  std::vector<std::vector<int>> marks;  // per host thread, per node: -1 outside a lookup scope
  // device copies of the IL structure (phase-B kernel)
  int* d_il_row = nullptr;
  int* d_il = nullptr;
  double** d_far = nullptr;
  int* d_capr = nullptr;
  int* d_il_ptr = nullptr;
  int* d_il_T = nullptr;
  double** d_M2M = nullptr;
  double** d_L2L = nullptr;
  // device copies of the near structure (Schur scatter kernel)
  int* d_nbr_ptr = nullptr;
  int* d_nbr = nullptr;
  int* d_slot_ptr = nullptr;
  int* d_n = nullptr;
  double** d_nb[3] = {nullptr, nullptr, nullptr};
  int slot(int p, int q) const {
    if (p == q) return slot_ptr[p];
    const int* b = LL->nbr.data() + LL->nbr_ptr[p];
    const int* e = LL->nbr.data() + LL->nbr_ptr[p + 1];
    const int* it = std::lower_bound(b, e, q);
    if (it == e || *it != q) return -1;
    return slot_ptr[p] + 1 + (int)(it - b);
  }
  int farix(int a, int b) const {
    const int* s = LL->il.data() + LL->il_ptr[a];
    const int* e = LL->il.data() + LL->il_ptr[a + 1];
    const int* it = std::lower_bound(s, e, b);
    if (it == e || *it != b) return -1;
    return (int)(it - LL->il.data());
  }
  bool is_near(int p, int q) const { return p == q || slot(p, q) >= 0; }
  int dim(int q) const { return elim[q] ? r[q] : n[q]; }  // current variable of q: x_q or y_q
};

struct Counter {
  double gemm = 0, inv = 0, qr = 0, svd = 0, lu = 0;
  void add_gemm(const std::vector<GemmDesc>& v) {
    for (auto& d : v) gemm += 2.0 * d.m * d.n * d.k;
  }
  double total() const { return gemm + inv + qr + svd + lu; }
};

// One recompression event (Algorithm 1's compression of the fill-ins at relative
// accuracy eps, Sec. 5.1; weighted as in Sec. 2.3's re-basing): new orthonormal
// row basis (P2M) and column basis (L2P) of a live node from the SVDs of the
// weighted old basis stacked with the far fill-ins.
struct Event {
  int q = 0;
  int r_old = 0, n = 0;
  std::vector<Blk> z[2];   // weighting blocks, logical rows x r_old
  Blk b[2];                // old basis as r_old x n (side 1: L2P^T)
  std::vector<Blk> f[2];   // fill rows, logical rows x n
  int nominal_rows[2] = {0, 0};
  double* V[2] = {nullptr, nullptr};
  double* sig[2] = {nullptr, nullptr};
  int avail[2] = {0, 0};
  int k = 0;
  double* T = nullptr;   // r_old x k
  double* Tp = nullptr;  // k x r_old
  int64_t key = 0;
  int event_no = 0;
  size_t sig_off[2] = {0, 0};
  int* kdev[2] = {nullptr, nullptr};
  int trigger = -1;  // eliminated neighbour whose fill-ins caused the event (-1: level start)
  float feat[IFMM_MLP_IN];
  int kcap = 0;      // learned cap of the pivoted QR (0: none)
  // what is needed to redo one side without the cap
  int gw_idx[2] = {-1, -1};
  int cf_first[2] = {0, 0}, cf_count[2] = {0, 0};
  QrcpDesc qd[2];
  SvdRtDesc sd[2];
  bool has_qd[2] = {false, false};
  bool rnd[2] = {false, false};  // randomized range finder (learned mode)
  double* Y[2] = {nullptr, nullptr};
  int my[2] = {0, 0};
  int zq = -1;  // >= 0: weight stacks gathered on the device for node zq (z lists unused)
  int mzd = 0;  //   their height
};

struct Factorizer {
  ifmm_fact& F;
  const ifmm_tree& T;
  cudaStream_t s;
  DescStage st;
  // Per-color scratch, two arenas used by alternate colors: a color's phase B/C
  // is issued after the next color's phase A (see run), so its buffers must
  // outlive that color's reset.
  DeviceArena scratch_buf[2];
  int scratch_sel = 0;
  DeviceArena& scratch() { return scratch_buf[scratch_sel]; }
  DeviceArena levelmem;
  int p, rc, maxrank;
  int prec = P64;  // arithmetic of Schur GEMMs and recompression (pivots stay FP64)
  int gprec = P64; // arithmetic of the Schur-complement GEMMs (P16 in the BF16 mode)
  double* m2m_tab = nullptr;
  double* m2l_tab = nullptr;
  std::unordered_map<int64_t, int> replay;
  std::vector<int> event_count;
  Counter cnt;
  // descriptor lists rebuilt for every color; members so that their capacity
  // survives from one color to the next (cleared before each use)
  struct Lists {
    std::vector<CopyDesc> cz, cpi, cg, sc, bc1, bc2, cc, cb;
    std::vector<QrDesc> qz;
    std::vector<QrcpDesc> qp;
    std::vector<GemmDesc> gw, gx, gf, b1, b2, c1, c2, gt;
    std::vector<SvdRtDesc> sr;
    std::vector<InvDesc> inv;
    std::vector<int> tl, tlf;
    std::vector<ZGatherDesc> zg;
    std::vector<ScatterDesc> scat;
    std::vector<unsigned char> el8;
    std::vector<const double*> tn, tpn;
  } L;
  template <class V>
  static V& fresh(V& v) {
    v.clear();
    return v;
  }
  int* d_info = nullptr;
  int info_cap = 0;
  std::vector<double*> pinned_sig;
  double t_wait = 0;
  float* d_mlp = nullptr;  // rank-predictor weights on the device (learned mode)
  double n_learned = 0, n_capped = 0, n_fallback = 0, qrcp_steps = 0;
  // host wall time of a factorization phase, accumulated into a stat
  void phase(const char* name, std::chrono::steady_clock::time_point& t) {
    const auto now = std::chrono::steady_clock::now();
    const double dt = std::chrono::duration<double>(now - t).count();
    F.stat_add(name, dt);
    F.stat_add(std::string(name) + "_L" + std::to_string(cur_level), dt);
    t = now;
  }
  int cur_level = 0;
  bool in_init = false;  // run_events called for a level's initial recompression
  const char* ev_tag(const char* part) {
    static thread_local std::string name;
    name = std::string(in_init ? "host_ev0_" : "host_ev_") + part;
    return name.c_str();
  }
  void wait() {
    auto a = std::chrono::steady_clock::now();
    CK(cudaStreamSynchronize(s));
    t_wait += std::chrono::duration<double>(std::chrono::steady_clock::now() - a).count();
  }

  Factorizer(ifmm_fact& f, cudaStream_t stream) : F(f), T(*f.t), s(stream) {
    st.stream = s;
    p = F.p;
    rc = F.rc;
    maxrank = F.o.max_rank > 0 ? F.o.max_rank : 256 * kernel_dof(F.k);
    prec = F.o.precision == IFMM_PREC_FP64 ? P64 : P32;
    gprec = F.o.precision == IFMM_PREC_BF16 ? P16 : prec;
    if (F.o.rank_mode == IFMM_RANK_LEARNED) {
      IFMM_REQUIRE(F.o.mlp != nullptr, IFMM_EINVAL, "learned rank mode needs the MLP weights");
      CK(cudaMalloc(&d_mlp, sizeof(float) * IFMM_MLP_NWEIGHTS));
      CK(cudaMemcpy(d_mlp, F.o.mlp, sizeof(float) * IFMM_MLP_NWEIGHTS, cudaMemcpyHostToDevice));
    }
    if (F.o.rank_mode == IFMM_RANK_REPLAY) {
      IFMM_REQUIRE(F.o.replay != nullptr || F.o.replay_len == 0, IFMM_EINVAL, "replay table is NULL");
      for (int64_t e = 0; e < F.o.replay_len; ++e) {
        const int32_t* qd = F.o.replay + 4 * e;
        replay[key3(qd[0], qd[1], qd[2])] = qd[3];
      }
    }
  }

  void sync() {
    CK(cudaStreamSynchronize(s));
    st.reset();
  }

  // Truncation threshold of the pivoted QR that precedes each SVD, relative to
  // the largest column norm: far enough below eps (divided by sqrt(n), which
  // bounds sigma_max of the discarded part) that the eps-rank subspace is kept
  // to well within the FP64 parity tolerance; in FP32 about two units of
  // roundoff.
  double tau_rel(int n) const {
    const double floor64 = 4.0 * std::max(n, 1) * std::ldexp(1.0, -52);
    if (prec == P32) return std::max(0.1 * F.o.eps, 2.0 * std::ldexp(1.0, -24));
    return std::max(F.o.eps > 0 ? 1e-4 * F.o.eps / std::sqrt((double)std::max(n, 1)) : 0.0, floor64);
  }

  // ------------------------------------------------------------------ ranks
  static int kept(const std::vector<double>& sig, int avail, int rows, int cols, double eps) {
    if (avail <= 0 || sig.empty() || !(sig[0] > 0.0)) return 0;
    const double thr = eps > 0.0 ? eps * sig[0] : (double)std::max(rows, cols) * std::ldexp(1.0, -52) * sig[0];
    int k = 0;
    for (int j = 0; j < avail && j < (int)sig.size(); ++j)
      if (sig[j] > thr) ++k;
    return k;
  }

  // ------------------------------------------------------------------ events
  // Runs the SVD stage of a batch of events, reads the singular values back,
  // picks the ranks, and leaves T, T' and the new bases in place.  P2M_out /
  // L2P_out / their lds give where the new bases go; the old bases are read
  // from ev.b before they are overwritten.
  void run_events(std::vector<Event>& evs, Work& W, const std::vector<double*>& P2M_out,
                  const std::vector<double*>& L2P_out, const std::vector<int>& P2M_ld, const std::vector<int>& L2P_ld,
                  std::vector<InvDesc>* inv_check, int n_inv, const ZTables* zt = nullptr) {
    auto tq = std::chrono::steady_clock::now();
    auto& cz = fresh(L.cz);
    auto& zg = fresh(L.zg);
    auto& qz = fresh(L.qz);
    auto& qp = fresh(L.qp);
    auto& gw = fresh(L.gw);
    auto& sr = fresh(L.sr);
    // heights of every event's weight stack (mz) and fill rows (mf), per side;
    // the events are split over host threads
    const int nevs = (int)evs.size();
    const int nthv = host_threads(nevs);
    std::vector<int> mzs(2 * (size_t)nevs), mfs(2 * (size_t)nevs);
    parallel_ranges(nthv, [&](int t) {
      const int x0 = (int)((long)nevs * t / nthv), x1 = (int)((long)nevs * (t + 1) / nthv);
      for (int x = x0; x < x1; ++x) {
        Event& ev = evs[x];
        for (int side = 0; side < 2; ++side) {
          int mz = 0;
          if (ev.zq >= 0)
            mz = ev.mzd;
          else
            for (auto& z : ev.z[side]) mz += z.rows;
          int mf = 0;
          for (auto& f : ev.f[side]) mf += f.rows;
          mzs[2 * (size_t)x + side] = mz;
          mfs[2 * (size_t)x + side] = mf;
        }
        ev.feat[5] = (float)(ev.r_old / 64.0);
        ev.feat[6] = (float)(mfs[2 * (size_t)x] / 1024.0);
      }
    });
    // learned mode: predicted rank of every event -> width of its sketch
    const bool learned = d_mlp && F.o.eps > 0.0;
    // a side is sketched when its predicted width is below this fraction of
    // the block's columns (IFMM_LEARNED_SKETCH_FRAC, read per factorization;
    // default 3/4), else it takes the exact path directly
    const double sketch_frac = [] {
      const char* e = getenv("IFMM_LEARNED_SKETCH_FRAC");
      const double f = e ? atof(e) : 0.75;
      return f > 0.0 && f <= 1.0 ? f : 0.75;
    }();
    if (learned && !evs.empty()) {
      std::vector<float> feat(evs.size() * IFMM_MLP_IN);
      for (size_t e = 0; e < evs.size(); ++e)
        memcpy(&feat[e * IFMM_MLP_IN], evs[e].feat, sizeof(float) * IFMM_MLP_IN);
      float* dx = (float*)scratch().alloc(feat.size() / 2 + 1);
      float* dy = (float*)scratch().alloc(evs.size() / 2 + 1);
      CK(cudaMemcpyAsync(dx, feat.data(), sizeof(float) * feat.size(), cudaMemcpyHostToDevice, s));
      float* dwk = (float*)scratch().alloc(mlp_predict_floats((int)evs.size()) / 2 + 1);
      mlp_predict_device(d_mlp, dx, dy, (int)evs.size(), s, dwk);
      float* hpred = (float*)st.host_alloc(sizeof(float) * evs.size());
      CK(cudaMemcpyAsync(hpred, dy, sizeof(float) * evs.size(), cudaMemcpyDeviceToHost, s));
      wait();
      const std::vector<float> pred(hpred, hpred + evs.size());
      for (size_t e = 0; e < evs.size(); ++e) {
        // sketch width: predicted rank plus oversampling
        const double k = std::max(0.0, (double)pred[e]) * 64.0;
        evs[e].kcap = std::max(1, (int)std::ceil(k) + 8);
        n_learned += 1;
      }
    }
    // contiguous readback buffers: singular values, truncation counts, tails
    size_t sig_total = 0;
    for (auto& ev : evs) sig_total += 2 * (size_t)ev.n;
    double* sig_all = scratch().alloc(std::max<size_t>(sig_total, 1));
    int* kall = (int*)scratch().alloc(evs.size() + 1);
    double* tail_all = scratch().alloc(2 * evs.size() + 1);
    // Placement, in event order (serial, O(events)): each side's spectrum
    // offset, its kind (0: empty block; 1: no rows, one zero fill of its
    // spectrum; 2: recompressed), its scratch (Z, Y, V, work, jp carved from one
    // allocation in the arena's 256-byte granules) and its first cf entry.
    auto rup = [](size_t x) { return (x + 31) & ~(size_t)31; };
    size_t sig_off = 0, woff = 0, cfn = 0;
    std::vector<int64_t> cfat(2 * (size_t)nevs, -1);  // first cf entry of the side
    std::vector<int> cfmw(2 * (size_t)nevs, 0);       // Y row of its first fill block
    std::vector<char> cfzero(2 * (size_t)nevs, 0);
    std::vector<char> kind(2 * (size_t)nevs, 0);
    std::vector<size_t> wat(2 * (size_t)nevs, 0);
    for (size_t e = 0; e < evs.size(); ++e) {
      Event& ev = evs[e];
      const int n = ev.n, r0 = ev.r_old;
      for (int side = 0; side < 2; ++side) {
        const size_t j = 2 * e + side;
        const int mz = mzs[j], mf = mfs[j];
        ev.sig_off[side] = sig_off;
        sig_off += n;
        if (n == 0) continue;
        const bool pathA = (n <= r0);
        const int mw = (mz == 0 || r0 == 0) ? 0 : (pathA ? mz : std::min(mz, r0));
        const int my = mw + mf;
        if (my == 0) {
          kind[j] = 1;
          cfat[j] = (int64_t)cfn++;
          cfzero[j] = 1;
          continue;
        }
        kind[j] = 2;
        cfat[j] = (int64_t)cfn;
        cfmw[j] = mw;
        cfn += ev.f[side].size();
        wat[j] = woff;
        woff += (mw > 0 ? rup((size_t)mz * r0) : 0) + rup((size_t)my * n) + 2 * rup((size_t)n * n) + rup((size_t)n / 2 + 1);
      }
    }
    double* wbase = woff ? scratch().alloc(woff) : nullptr;
    // Descriptors, by host threads over event ranges into local lists joined in
    // event order (the launch order of a serial loop).
    struct EvLists {
      std::vector<CopyDesc> cz;
      std::vector<ZGatherDesc> zg;
      std::vector<QrDesc> qz;
      std::vector<GemmDesc> gw;
      std::vector<QrcpDesc> qp;
      std::vector<SvdRtDesc> sr;
      double qr = 0.0, svd = 0.0;
    };
    std::vector<EvLists> evl(nthv);
    parallel_ranges(nthv, [&](int t) {
      const int x0 = (int)((long)nevs * t / nthv), x1 = (int)((long)nevs * (t + 1) / nthv);
      EvLists o;
      for (int e = x0; e < x1; ++e) {
        Event& ev = evs[e];
        const int n = ev.n, r0 = ev.r_old;
        for (int side = 0; side < 2; ++side) {
          const size_t j = 2 * (size_t)e + side;
          const int mz = mzs[j], mf = mfs[j];
          ev.nominal_rows[side] = r0 + mf;
          ev.avail[side] = std::min(r0 + mf, n);
          ev.V[side] = nullptr;
          ev.sig[side] = sig_all + ev.sig_off[side];
          ev.kdev[side] = kall + j;
          if (kind[j] == 0) continue;
          if (kind[j] == 1) {
            ev.avail[side] = 0;
            continue;
          }
          const bool pathA = (n <= r0);
          const int mw = (mz == 0 || r0 == 0) ? 0 : (pathA ? mz : std::min(mz, r0));
          const int my = mw + mf;
          // the pieces, each registered for the bounds checks (IFMM_CHECK)
          double* w = wbase + wat[j];
          auto piece = [&](size_t cnt) {
            double* p = w;
            registry().add(p, sizeof(double) * cnt);
            w += rup(cnt);
            return p;
          };
          double* Z = nullptr;
          if (mw > 0) {
            Z = piece((size_t)mz * r0);
            if (ev.zq >= 0) {
              IFMM_REQUIRE(zt, IFMM_EINVAL, "internal: device weight stack without tables");
              o.zg.push_back(ZGatherDesc{Z, mz, ev.zq, side, 0});
            } else {
              int off = 0;
              for (auto& z : ev.z[side]) {
                o.cz.push_back(cpy(z.p, z.ld, Z + off, mz, z.rows, z.cols, 1.0, 0.0, z.trans));
                off += z.rows;
              }
            }
            if (!pathA) {
              o.qz.push_back(QrDesc{Z, mz, mz, r0});
              const double mn = std::min(mz, r0);
              o.qr += 2.0 * mz * r0 * (double)r0 - 2.0 * (mn * mn * mn) / 3.0;
            }
          }
          double* Y = piece((size_t)my * n);
          if (mw > 0) {
            const Blk& B = ev.b[side];
            // W = Z * B (path A) or R_Z * B (path B); B logical r0 x n
            ev.gw_idx[side] = (int)o.gw.size();  // made global after the join
            o.gw.push_back(gmm(Z, mz, 0, B.p, B.ld, B.trans, Y, my, mw, n, r0, 1.0, 0.0));
          }
          ev.cf_first[side] = (int)cfat[j];
          ev.cf_count[side] = (int)ev.f[side].size();
          ev.V[side] = piece((size_t)n * n);
          double* work = piece((size_t)n * n);
          int* jp = (int*)piece((size_t)n / 2 + 1);
          QrcpDesc qd;
          qd.A = Y;
          qd.ld = my;
          qd.m = my;
          qd.n = n;
          qd.tau_rel = tau_rel(n);
          qd.jpvt = jp;
          qd.kout = ev.kdev[side];
          qd.kcap = 0;
          qd.pad = 0;
          qd.rb = 0;
          qd.rs = 0;
          qd.tail = tail_all + j;
          ev.qd[side] = qd;
          ev.has_qd[side] = true;
          ev.Y[side] = Y;
          ev.my[side] = my;
          // learned mode: a randomized range finder at the predicted rank when it
          // is clearly narrower than the block; otherwise the exact path
          ev.rnd[side] = learned && ev.kcap < sketch_frac * n && ev.kcap < my;
          if (!ev.rnd[side]) o.qp.push_back(qd);
          SvdRtDesc sd;
          sd.A = Y;
          sd.ld = my;
          sd.n = n;
          sd.jpvt = jp;
          sd.kin = ev.kdev[side];
          sd.V = ev.V[side];
          sd.ldv = n;
          sd.pad = 0;
          sd.sig = ev.sig[side];
          sd.work = work;
          if (!ev.rnd[side]) o.sr.push_back(sd);
          ev.sd[side] = sd;
          const double mm = std::max(my, n), nn = std::min(my, n);
          o.qr += 2.0 * mm * nn * nn - 2.0 * nn * nn * nn / 3.0;
          const double ms = std::min(ev.nominal_rows[side], n);
          o.svd += 6.0 * std::max(ev.nominal_rows[side], n) * (ms * ms) + 20.0 * (ms * ms * ms);
        }
      }
      evl[t] = std::move(o);
    });
    for (int t = 0; t < nthv; ++t) {
      const int x0 = (int)((long)nevs * t / nthv), x1 = (int)((long)nevs * (t + 1) / nthv);
      const int g0 = (int)gw.size();
      for (int e = x0; e < x1; ++e)
        for (int side = 0; side < 2; ++side)
          if (evs[e].gw_idx[side] >= 0 && kind[2 * (size_t)e + side] == 2) evs[e].gw_idx[side] += g0;
      EvLists& o = evl[t];
      cz.insert(cz.end(), o.cz.begin(), o.cz.end());
      zg.insert(zg.end(), o.zg.begin(), o.zg.end());
      qz.insert(qz.end(), o.qz.begin(), o.qz.end());
      gw.insert(gw.end(), o.gw.begin(), o.gw.end());
      qp.insert(qp.end(), o.qp.begin(), o.qp.end());
      sr.insert(sr.end(), o.sr.begin(), o.sr.end());
      cnt.qr += o.qr;
      cnt.svd += o.svd;
    }
    // The cf copies in event order, sorted (stably) into the small and the large
    // ones straight in the pinned staging buffer: per thread, how many of each;
    // then each thread writes its own, at the exclusive prefix of the counts.
    std::vector<size_t> cf_ns(nthv + 1, 0), cf_nb(nthv + 1, 0);
    auto cf_entry = [&](const Event& ev, int side, size_t j, const Blk* f, int off) {
      return cfzero[j] ? cpy(nullptr, 0, ev.sig[side], ev.n, ev.n, 1)
                       : cpy(f->p, f->ld, ev.Y[side] + off, ev.my[side], f->rows, f->cols, 1.0, 0.0, f->trans);
    };
    auto cf_each = [&](int t, auto&& put) {
      const int x0 = (int)((long)nevs * t / nthv), x1 = (int)((long)nevs * (t + 1) / nthv);
      for (int x = x0; x < x1; ++x) {
        const Event& ev = evs[x];
        for (int side = 0; side < 2; ++side) {
          const size_t j = 2 * (size_t)x + side;
          if (cfat[j] < 0) continue;
          if (cfzero[j]) {
            put(cf_entry(ev, side, j, nullptr, 0));
            continue;
          }
          int off = cfmw[j];
          for (auto& f : ev.f[side]) {
            put(cf_entry(ev, side, j, &f, off));
            off += f.rows;
          }
        }
      }
    };
    parallel_ranges(nthv, [&](int t) {
      size_t a = 0, b = 0;
      cf_each(t, [&](const CopyDesc& c) { ++(copy_is_small(c) ? a : b); });
      cf_ns[t + 1] = a;
      cf_nb[t + 1] = b;
    });
    for (int t = 0; t < nthv; ++t) {
      cf_ns[t + 1] += cf_ns[t];
      cf_nb[t + 1] += cf_nb[t];
    }
    IFMM_REQUIRE(cf_ns[nthv] + cf_nb[nthv] == cfn, IFMM_EINVAL, "internal: fill copy count");
    CopyDesc* cf_h = cfn ? (CopyDesc*)st.host_alloc(sizeof(CopyDesc) * cfn) : nullptr;
    parallel_ranges(nthv, [&](int t) {
      size_t a = cf_ns[t], b = cf_ns[nthv] + cf_nb[t];
      cf_each(t, [&](const CopyDesc& c) { cf_h[copy_is_small(c) ? a++ : b++] = c; });
    });
    phase(ev_tag("build"), tq);
    CK(cudaMemsetAsync(kall, 0, sizeof(int) * (evs.size() * 2 + 0), s));
    CK(cudaMemsetAsync(tail_all, 0, sizeof(double) * (evs.size() * 2 + 1), s));
    launch_copy(st, cz);
    if (!zg.empty()) launch_zgather(st, zg, *zt);
    launch_qr(st, qz, prec);
    cnt.add_gemm(gw);
    launch_gemm(st, gw, prec);
    launch_copy_sorted(st, cf_h, cf_ns[nthv], cf_nb[nthv]);
    launch_qrcp(st, qp, prec);
    launch_svd_rt(st, sr, prec);
    // randomized range finder (Halko, Martinsson, Tropp) at the predicted rank s:
    // Z = Y^T Omega, Q = orth(Z), B = Y Q, SVD of B -> V = Q V_B; residual
    // E = Y - B Q^T, whose Frobenius norm bounds what the sketch missed
    double* enorm_all = scratch().alloc(2 * evs.size() + 1);
    double* ynorm_all = scratch().alloc(2 * evs.size() + 1);
    {
      std::vector<SketchDesc> sk;
      std::vector<GemmDesc> g1, g2, g3, g4;
      std::vector<SvdRtDesc> so, sb;
      std::vector<QrcpDesc> qb;
      std::vector<CopyDesc> ce, cz0;
      std::vector<FrobDesc> fr;
      std::vector<int> widths;
      std::vector<int*> wdev;
      int* sarr = (int*)scratch().alloc(evs.size() + 1);
      for (size_t e = 0; e < evs.size(); ++e)
        for (int side = 0; side < 2; ++side) {
          Event& ev = evs[e];
          if (!ev.rnd[side]) continue;
          const int n = ev.n, my = ev.my[side], sw = std::min(ev.kcap, n);
          double* Om = scratch().alloc((size_t)my * sw);
          double* Zs = scratch().alloc((size_t)n * sw);
          double* Q = scratch().alloc((size_t)n * n);
          double* qs = scratch().alloc(n);
          double* qw = scratch().alloc((size_t)n * n);
          double* Bm = scratch().alloc((size_t)my * sw);
          double* VB = scratch().alloc((size_t)sw * sw);
          double* bw = scratch().alloc((size_t)sw * sw);
          double* E = scratch().alloc((size_t)my * n);
          int* jpb = (int*)scratch().alloc((size_t)sw / 2 + 1);
          int* sdev = sarr + widths.size();
          widths.push_back(sw);
          sk.push_back(SketchDesc{Om, my, sw, (unsigned long long)(F.o.seed * 0x100000001B3ull + (uint64_t)ev.key * 2 + side)});
          g1.push_back(gmm(ev.Y[side], my, 1, Om, my, 0, Zs, n, n, sw, my, 1.0, 0.0));  // Z = Y^T Omega
          SvdRtDesc o;
          o.A = Zs;
          o.ld = n;
          o.n = n;
          o.jpvt = nullptr;
          o.kin = sdev;
          o.V = Q;
          o.ldv = n;
          o.pad = 0;
          o.sig = qs;
          o.work = qw;
          so.push_back(o);                                                                  // Q = orth(Z)
          g2.push_back(gmm(ev.Y[side], my, 0, Q, n, 0, Bm, my, my, sw, n, 1.0, 0.0));       // B = Y Q
          QrcpDesc qd = ev.qd[side];
          qd.A = Bm;
          qd.ld = my;
          qd.m = my;
          qd.n = sw;
          qd.jpvt = jpb;
          qb.push_back(qd);
          SvdRtDesc b = ev.sd[side];
          b.A = Bm;
          b.ld = my;
          b.n = sw;
          b.jpvt = jpb;
          b.kin = ev.kdev[side];
          b.V = VB;
          b.ldv = sw;
          b.sig = ev.sig[side];
          b.work = bw;
          cz0.push_back(cpy(nullptr, 0, ev.sig[side], n, n, 1));
          sb.push_back(b);
          g3.push_back(gmm(Q, n, 0, VB, sw, 0, ev.V[side], n, n, sw, sw, 1.0, 0.0));      // V = Q V_B
          ce.push_back(cpy(ev.Y[side], my, E, my, my, n));
          g4.push_back(gmm(Bm, my, 0, Q, n, 1, E, my, my, n, sw, -1.0, 1.0));              // E = Y - B Q^T
          fr.push_back(FrobDesc{E, my, my, n, enorm_all + 2 * e + side});
          fr.push_back(FrobDesc{ev.Y[side], my, my, n, ynorm_all + 2 * e + side});
        }
      if (!widths.empty()) {
        CK(cudaMemcpyAsync(sarr, widths.data(), sizeof(int) * widths.size(), cudaMemcpyHostToDevice, s));
        // B = Y Q is needed twice (pivoted QR destroys it): keep the SVD on a copy
        launch_sketch(st, sk);
        cnt.add_gemm(g1);
        launch_gemm(st, g1, prec);
        launch_svd_rt(st, so, prec);
        cnt.add_gemm(g2);
        launch_gemm(st, g2, prec);
        launch_copy(st, ce);
        cnt.add_gemm(g4);
        launch_gemm(st, g4, prec);
        launch_frob(st, fr);
        launch_copy(st, cz0);
        launch_qrcp(st, qb, prec);
        launch_svd_rt(st, sb, prec);
        cnt.add_gemm(g3);
        launch_gemm(st, g3, prec);
      }
    }
    // read back singular values, truncation counts and pivot status
    std::vector<double> hsig(sig_total);
    std::vector<int> hk(2 * evs.size(), 0);
    double* hp = nullptr;
    int* hkp = nullptr;
    if (sig_total) {
      hp = (double*)st.host_alloc(sig_total * sizeof(double));
      CK(cudaMemcpyAsync(hp, sig_all, sizeof(double) * sig_total, cudaMemcpyDeviceToHost, s));
    }
    if (!evs.empty()) {
      hkp = (int*)st.host_alloc(sizeof(int) * 2 * evs.size());
      CK(cudaMemcpyAsync(hkp, kall, sizeof(int) * 2 * evs.size(), cudaMemcpyDeviceToHost, s));
    }
    std::vector<int> hinfo(n_inv, 0);
    int* hi = nullptr;
    if (n_inv) {
      hi = (int*)st.host_alloc(sizeof(int) * n_inv);
      CK(cudaMemcpyAsync(hi, d_info, sizeof(int) * n_inv, cudaMemcpyDeviceToHost, s));
    }
    // learned mode: the sketches' residual and input norms, in the same readback
    double* hen = nullptr;
    if (learned && !evs.empty()) {
      hen = (double*)st.host_alloc(sizeof(double) * 4 * evs.size());
      CK(cudaMemcpyAsync(hen, enorm_all, sizeof(double) * 2 * evs.size(), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hen + 2 * evs.size(), ynorm_all, sizeof(double) * 2 * evs.size(), cudaMemcpyDeviceToHost,
                         s));
    }
    phase(ev_tag("launch"), tq);
    wait();
    phase(ev_tag("wait"), tq);
    if (sig_total) memcpy(hsig.data(), hp, sig_total * sizeof(double));
    if (!evs.empty()) memcpy(hk.data(), hkp, sizeof(int) * 2 * evs.size());
    if (n_inv) memcpy(hinfo.data(), hi, sizeof(int) * n_inv);
    st.reset();
    for (int i = 0; i < n_inv; ++i)
      IFMM_REQUIRE(hinfo[i] == 0, IFMM_ESINGULAR, "singular pivot block at level " + std::to_string(W.kappa));
    (void)inv_check;
    if (learned && !evs.empty()) {
      // a-posteriori check of every sketch: ||Y - B Q^T||_F (>= the 2-norm of
      // what the range finder missed) must be <= eps * sigma_1; sides that fail
      // run the exact path on Y, which the randomized path left untouched
      const std::vector<double> en(hen, hen + 2 * evs.size()), yn(hen + 2 * evs.size(), hen + 4 * evs.size());
      // below 16 units of roundoff of the arithmetic (times ||Y||_F) no
      // recompression in that arithmetic can certify anything
      const double unit = prec == P32 ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
      std::vector<QrcpDesc> rqp;
      std::vector<SvdRtDesc> rsr;
      std::vector<std::pair<size_t, int>> redo;
      for (size_t e = 0; e < evs.size(); ++e)
        for (int side = 0; side < 2; ++side) {
          Event& ev = evs[e];
          if (!ev.rnd[side]) continue;
          n_capped += 0.5;
          const double s1 = hsig[ev.sig_off[side]];
          if (en[2 * e + side] <= std::max(F.o.eps * s1, 16.0 * unit * yn[2 * e + side])) continue;
          redo.push_back({e, side});
          rqp.push_back(ev.qd[side]);
          rsr.push_back(ev.sd[side]);
        }
      if (!redo.empty()) {
        n_fallback += (double)redo.size() * 0.5;
        launch_qrcp(st, rqp, prec);
        launch_svd_rt(st, rsr, prec);
        // one readback of every count and spectrum (the redone ones changed)
        double* hp2 = (double*)st.host_alloc(sizeof(double) * std::max<size_t>(sig_total, 1));
        int* hk2 = (int*)st.host_alloc(sizeof(int) * 2 * evs.size());
        if (sig_total) CK(cudaMemcpyAsync(hp2, sig_all, sizeof(double) * sig_total, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hk2, kall, sizeof(int) * 2 * evs.size(), cudaMemcpyDeviceToHost, s));
        wait();
        for (auto& rd : redo) {
          const Event& ev = evs[rd.first];
          memcpy(hsig.data() + ev.sig_off[rd.second], hp2 + ev.sig_off[rd.second], sizeof(double) * ev.n);
          hk[2 * rd.first + rd.second] = hk2[2 * rd.first + rd.second];
        }
        st.reset();
      }
    }
    for (size_t e = 0; e < evs.size(); ++e)
      for (int side = 0; side < 2; ++side)
        if (evs[e].V[side]) {
          evs[e].avail[side] = std::min(evs[e].avail[side], hk[2 * e + side]);
          qrcp_steps += hk[2 * e + side];
        }
    // choose ranks (max of the row and column counts, both sides share it)
    for (auto& ev : evs) {
      std::vector<double> sg[2];
      for (int side = 0; side < 2; ++side)
        if (ev.V[side]) sg[side].assign(hsig.begin() + ev.sig_off[side], hsig.begin() + ev.sig_off[side] + ev.n);
      const int kr = kept(sg[0], ev.avail[0], ev.nominal_rows[0], ev.n, F.o.eps);
      const int kc = kept(sg[1], ev.avail[1], ev.nominal_rows[1], ev.n, F.o.eps);
      int k = std::min(std::max(kr, kc), std::min(ev.avail[0], ev.avail[1]));
      if (F.o.rank_mode == IFMM_RANK_REPLAY) {
        auto it = replay.find(ev.key);
        IFMM_REQUIRE(it != replay.end(), IFMM_EINVAL, "replay table misses an event");
        k = it->second;
        IFMM_REQUIRE(k >= 0 && k <= std::min(ev.avail[0], ev.avail[1]), IFMM_EINVAL, "replayed rank out of range");
      }
      // the blocks of q were sized for at most capr[q] = min(n_q, max_rank)
      // columns: a larger rank would break the eps guarantee if cut, so it is an error
      IFMM_REQUIRE(k <= W.capr[ev.q], IFMM_ERANK,
                   "level " + std::to_string(W.kappa) + " node " + std::to_string(ev.q) + " needs rank " +
                       std::to_string(k) + " above max_rank " + std::to_string(maxrank));
      ev.k = k;
      F.rank_log.push_back({W.kappa, ev.q, ev.event_no, k});
      F.event_feat.insert(F.event_feat.end(), ev.feat, ev.feat + IFMM_MLP_IN);
    }
    phase(ev_tag("ranks"), tq);
    // T = P2M_old V_row[:, :k], T' = V_col[:, :k]^T L2P_old, then the new bases
    auto& gt = fresh(L.gt);
    auto& cb = fresh(L.cb);
    for (size_t e = 0; e < evs.size(); ++e) {
      Event& ev = evs[e];
      const int k = ev.k, n = ev.n, r0 = ev.r_old;
      ev.T = scratch().alloc((size_t)std::max(1, r0 * k));
      ev.Tp = scratch().alloc((size_t)std::max(1, r0 * k));
      if (k == 0) continue;
      // side 0: B = P2M_old (r0 x n); side 1: B = L2P_old^T
      if (r0 > 0) {
        gt.push_back(gmm(ev.b[0].p, ev.b[0].ld, ev.b[0].trans, ev.V[0], n, 0, ev.T, r0, r0, k, n, 1.0, 0.0));
        // T' = V_col[:, :k]^T * L2P_old  (L2P_old = (b[1])^T)
        gt.push_back(gmm(ev.V[1], n, 1, ev.b[1].p, ev.b[1].ld, ev.b[1].trans ? 0 : 1, ev.Tp, k, k, r0, n, 1.0, 0.0));
      }
      cb.push_back(cpy(ev.V[0], n, P2M_out[e], P2M_ld[e], k, n, 1.0, 0.0, 1));
      cb.push_back(cpy(ev.V[1], n, L2P_out[e], L2P_ld[e], n, k, 1.0, 0.0, 0));
    }
    cnt.add_gemm(gt);
    launch_gemm(st, gt, prec);
    launch_copy(st, cb);
    phase(ev_tag("tail"), tq);
  }

  Event make_event(Work& W, int q, int trigger = -1) {
    Event ev;
    ev.q = q;
    ev.event_no = event_count[q]++;
    ev.key = key3(W.kappa, q, ev.event_no);
    ev.trigger = trigger;
    // rank-predictor inputs: cell centre in [-1,1]^3, cell size and level, offset
    // to the eliminated neighbour, log10(eps)
    const LevelLists& LL = *W.LL;
    const double m = (double)((int64_t)1 << W.kappa);
    int l1 = 0;
    for (int d = 0; d < 3; ++d) {
      ev.feat[d] = (float)((LL.cells[3 * q + d] + 0.5) / m * 2.0 - 1.0);
      if (trigger >= 0) l1 += std::abs(LL.cells[3 * q + d] - LL.cells[3 * trigger + d]);
    }
    ev.feat[3] = (float)(W.n[q] / 256.0);          // block size n_q
    ev.feat[4] = (float)(W.kappa / 10.0);
    ev.feat[5] = (float)(W.r[q] / 64.0);           // current rank (set by set_event_sizes)
    ev.feat[6] = 0.f;                              // fill rows (set by set_event_sizes)
    ev.feat[7] = (float)(l1 / 3.0);                // offset to the eliminated neighbour, L1
    ev.feat[8] = (float)((F.o.eps > 0 ? std::log10(F.o.eps) : -16.0) / 10.0);
    return ev;
  }

  // ------------------------------------------------------------------ level start
  void init_level(Work& W, int kappa, Work* child) {
    const LevelLists& LL = T.lv[kappa];
    auto tq = std::chrono::steady_clock::now();
    W.kappa = kappa;
    W.LL = &LL;
    W.nn = LL.n;
    const int nn = LL.n;
    W.n.assign(nn, 0);
    if (!child) {
      for (int i = 0; i < nn; ++i) W.n[i] = kernel_dof(F.k) * (T.leaf_ptr[i + 1] - T.leaf_ptr[i]);
    } else {
      child->choff.assign(child->nn, 0);
      for (int a = 0; a < nn; ++a) {
        int off = 0;
        for (int c = LL.child_ptr[a]; c < LL.child_ptr[a + 1]; ++c) {
          const int ch = LL.child[c];
          child->choff[ch] = off;
          off += child->r[ch];
        }
        W.n[a] = off;
      }
    }
    W.capr.resize(nn);
    for (int i = 0; i < nn; ++i) W.capr[i] = std::min(W.n[i], maxrank);
    W.r.assign(nn, 0);
    W.elim.assign(nn, 0);
    event_count.assign(nn, 0);
    W.il_row.assign(LL.il.size(), 0);
    W.il_T.assign(LL.il.size(), -1);
    {
      const int nt = host_threads(nn);
      parallel_ranges(nt, [&](int t) {
        const int a0 = (int)((long)nn * t / nt), a1 = (int)((long)nn * (t + 1) / nt);
        for (int a = a0; a < a1; ++a)
          for (int e = LL.il_ptr[a]; e < LL.il_ptr[a + 1]; ++e) {
            W.il_row[e] = a;
            W.il_T[e] = W.farix(LL.il[e], a);
            IFMM_REQUIRE(W.il_T[e] >= 0, IFMM_EINVAL, "internal: interaction list not symmetric");
          }
      });
    }
    phase("host_init_lists", tq);
    // near slots
    W.slot_ptr.assign(nn + 1, 0);
    for (int i = 0; i < nn; ++i) W.slot_ptr[i + 1] = W.slot_ptr[i] + 1 + (LL.nbr_ptr[i + 1] - LL.nbr_ptr[i]);
    const int nslots = W.slot_ptr[nn];
    for (int s3 = 0; s3 < 3; ++s3) W.nb[s3].assign(nslots, nullptr);
    for (int i = 0; i < nn; ++i) {
      for (int k = 0; k <= LL.nbr_ptr[i + 1] - LL.nbr_ptr[i]; ++k) {
        const int q = k == 0 ? i : LL.nbr[LL.nbr_ptr[i] + k - 1];
        const size_t sz = (size_t)std::max(1, W.n[i]) * std::max(1, W.n[q]);
        const int sl = W.slot_ptr[i] + k;
        W.nb[0][sl] = F.persist.alloc(sz);
        if (k > 0) W.nb[1][sl] = F.persist.alloc(sz);
        W.nb[2][sl] = levelmem.alloc(sz);
      }
    }
    {
      W.d_nbr_ptr = (int*)levelmem.alloc_bytes(sizeof(int) * (nn + 1));
      W.d_nbr = (int*)levelmem.alloc_bytes(sizeof(int) * std::max<size_t>(1, LL.nbr.size()));
      W.d_slot_ptr = (int*)levelmem.alloc_bytes(sizeof(int) * (nn + 1));
      W.d_n = (int*)levelmem.alloc_bytes(sizeof(int) * std::max(1, nn));
      CK(cudaMemcpyAsync(W.d_nbr_ptr, LL.nbr_ptr.data(), sizeof(int) * (nn + 1), cudaMemcpyHostToDevice, s));
      if (!LL.nbr.empty())
        CK(cudaMemcpyAsync(W.d_nbr, LL.nbr.data(), sizeof(int) * LL.nbr.size(), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(W.d_slot_ptr, W.slot_ptr.data(), sizeof(int) * (nn + 1), cudaMemcpyHostToDevice, s));
      if (nn) CK(cudaMemcpyAsync(W.d_n, W.n.data(), sizeof(int) * nn, cudaMemcpyHostToDevice, s));
      for (int s3 = 0; s3 < 3; ++s3) {
        W.d_nb[s3] = (double**)levelmem.alloc_bytes(sizeof(double*) * std::max(1, nslots));
        if (nslots)
          CK(cudaMemcpyAsync(W.d_nb[s3], W.nb[s3].data(), sizeof(double*) * nslots, cudaMemcpyHostToDevice, s));
      }
    }
    W.far.assign(LL.il.size(), nullptr);
    {
      // one allocation for every far block of the level (256-byte granules, as
      // the arena's own), carved in IL order
      auto rup = [](size_t x) { return (x + 31) & ~(size_t)31; };
      size_t tot = 0;
      for (int a = 0; a < nn; ++a)
        for (int e = LL.il_ptr[a]; e < LL.il_ptr[a + 1]; ++e)
          tot += rup((size_t)std::max(1, W.capr[a]) * std::max(1, W.capr[LL.il[e]]));
      double* blk = tot ? levelmem.alloc(tot) : nullptr;
      size_t off = 0;
      for (int a = 0; a < nn; ++a)
        for (int e = LL.il_ptr[a]; e < LL.il_ptr[a + 1]; ++e) {
          W.far[e] = blk + off;
          off += rup((size_t)std::max(1, W.capr[a]) * std::max(1, W.capr[LL.il[e]]));
        }
    }
    {
      const size_t ne = std::max<size_t>(1, LL.il.size());
      W.d_il_row = (int*)levelmem.alloc_bytes(sizeof(int) * ne);
      W.d_il = (int*)levelmem.alloc_bytes(sizeof(int) * ne);
      W.d_far = (double**)levelmem.alloc_bytes(sizeof(double*) * ne);
      W.d_capr = (int*)levelmem.alloc_bytes(sizeof(int) * std::max(1, nn));
      if (!LL.il.empty()) {
        CK(cudaMemcpyAsync(W.d_il_row, W.il_row.data(), sizeof(int) * LL.il.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(W.d_il, LL.il.data(), sizeof(int) * LL.il.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(W.d_far, W.far.data(), sizeof(double*) * LL.il.size(), cudaMemcpyHostToDevice, s));
      }
      if (nn) CK(cudaMemcpyAsync(W.d_capr, W.capr.data(), sizeof(int) * nn, cudaMemcpyHostToDevice, s));
    }
    W.P2M.assign(nn, nullptr);
    W.L2P.assign(nn, nullptr);
    W.M2M.assign(nn, nullptr);
    W.L2L.assign(nn, nullptr);
    for (int i = 0; i < nn; ++i) {
      W.P2M[i] = levelmem.alloc((size_t)std::max(1, W.capr[i]) * std::max(1, W.n[i]));
      W.L2P[i] = levelmem.alloc((size_t)std::max(1, W.capr[i]) * std::max(1, W.n[i]));
      if (kappa > 2) {
        W.M2M[i] = levelmem.alloc((size_t)rc * std::max(1, W.capr[i]));
        W.L2L[i] = levelmem.alloc((size_t)rc * std::max(1, W.capr[i]));
      }
    }
    {
      const size_t ne = std::max<size_t>(1, LL.il.size());
      W.d_il_ptr = (int*)levelmem.alloc_bytes(sizeof(int) * (nn + 1));
      W.d_il_T = (int*)levelmem.alloc_bytes(sizeof(int) * ne);
      W.d_M2M = (double**)levelmem.alloc_bytes(sizeof(double*) * std::max(1, nn));
      W.d_L2L = (double**)levelmem.alloc_bytes(sizeof(double*) * std::max(1, nn));
      CK(cudaMemcpyAsync(W.d_il_ptr, LL.il_ptr.data(), sizeof(int) * (nn + 1), cudaMemcpyHostToDevice, s));
      if (!LL.il.empty())
        CK(cudaMemcpyAsync(W.d_il_T, W.il_T.data(), sizeof(int) * LL.il.size(), cudaMemcpyHostToDevice, s));
      if (nn) {
        CK(cudaMemcpyAsync(W.d_M2M, W.M2M.data(), sizeof(double*) * nn, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(W.d_L2L, W.L2L.data(), sizeof(double*) * nn, cudaMemcpyHostToDevice, s));
      }
    }
    phase("host_init_alloc", tq);
    // stage-0 near blocks and the initial bases (r_cheb columns / rows)
    scratch_sel = 0;
    scratch().reset();
    std::vector<double*> P2M0(nn), L2P0(nn);
    for (int i = 0; i < nn; ++i) {
      P2M0[i] = scratch().alloc((size_t)rc * std::max(1, W.n[i]));
      L2P0[i] = scratch().alloc((size_t)rc * std::max(1, W.n[i]));
    }
    if (!child) {
      std::vector<P2pDesc> pp;
      std::vector<InterpDesc> ip;
      std::vector<CopyDesc> ct;
      const double h = 0.5 * T.side / (double)((int64_t)1 << kappa);
      for (int i = 0; i < nn; ++i) {
        for (int k = 0; k <= LL.nbr_ptr[i + 1] - LL.nbr_ptr[i]; ++k) {
          const int q = k == 0 ? i : LL.nbr[LL.nbr_ptr[i] + k - 1];
          P2pDesc d;
          d.dst = W.nb[0][W.slot_ptr[i] + k];
          d.i0 = T.leaf_ptr[i];
          d.ni = T.leaf_ptr[i + 1] - T.leaf_ptr[i];
          d.j0 = T.leaf_ptr[q];
          d.nj = T.leaf_ptr[q + 1] - T.leaf_ptr[q];
          d.ld = W.n[i];
          d.same = (q == i);
          pp.push_back(d);
        }
        InterpDesc id;
        id.dst = P2M0[i];
        id.cx = T.origin[0] + (LL.cells[3 * i] + 0.5) * 2 * h;
        id.cy = T.origin[1] + (LL.cells[3 * i + 1] + 0.5) * 2 * h;
        id.cz = T.origin[2] + (LL.cells[3 * i + 2] + 0.5) * 2 * h;
        id.h = h;
        id.p0 = T.leaf_ptr[i];
        id.n = T.leaf_ptr[i + 1] - T.leaf_ptr[i];
        id.ld = rc;
        id.pad = 0;
        ip.push_back(id);
        ct.push_back(cpy(P2M0[i], rc, L2P0[i], W.n[i], W.n[i], rc, 1.0, 0.0, 1));
      }
      launch_p2p(st, pp, T.d_pts, (int)T.N, F.k);
      launch_interp(st, ip, T.d_pts, (int)T.N, p, kernel_dof(F.k));
      launch_copy(st, ct);
    } else {
      std::vector<CopyDesc> cc;
      const LevelLists& CL = *child->LL;
      for (int a = 0; a < nn; ++a) {
        for (int k = 0; k <= LL.nbr_ptr[a + 1] - LL.nbr_ptr[a]; ++k) {
          const int b = k == 0 ? a : LL.nbr[LL.nbr_ptr[a] + k - 1];
          double* dst = W.nb[0][W.slot_ptr[a] + k];
          for (int x = LL.child_ptr[a]; x < LL.child_ptr[a + 1]; ++x) {
            const int c = LL.child[x];
            for (int y = LL.child_ptr[b]; y < LL.child_ptr[b + 1]; ++y) {
              const int d = LL.child[y];
              const int sl = child->slot(c, d);
              const double* src;
              int ld;
              if (sl >= 0) {
                src = child->nb[2][sl];
                ld = child->n[c];
              } else {
                const int fx = child->farix(c, d);
                IFMM_REQUIRE(fx >= 0, IFMM_EINVAL, "internal: child pair neither near nor far");
                src = child->far[fx];
                ld = child->capr[c];
              }
              if (child->r[c] && child->r[d])
                cc.push_back(cpy(src, ld, dst + child->choff[c] + (long)child->choff[d] * W.n[a], W.n[a], child->r[c],
                                 child->r[d]));
            }
          }
        }
        for (int x = LL.child_ptr[a]; x < LL.child_ptr[a + 1]; ++x) {
          const int c = LL.child[x];
          if (!child->r[c]) continue;
          cc.push_back(cpy(child->M2M[c], rc, P2M0[a] + (long)child->choff[c] * rc, rc, rc, child->r[c]));
          cc.push_back(cpy(child->L2L[c], child->capr[c], L2P0[a] + child->choff[c], W.n[a], child->r[c], rc));
        }
      }
      (void)CL;
      launch_copy(st, cc);
    }
    phase("host_init_blocks", tq);
    // M2L translation table of this level
    const double h = 0.5 * T.side / (double)((int64_t)1 << kappa);
    m2l_tab = levelmem.alloc((size_t)343 * rc * rc);
    launch_m2l_table(s, m2l_tab, p, h, F.k);
    // initial recompression of every node (the leaf rank p^3 exceeds the
    // points of a leaf, Sec. 2.3)
    std::vector<Event> evs;
    std::vector<double*> po, lo;
    std::vector<int> pld, lld;
    auto off_index = [&](int a, int b) {
      const int dx = LL.cells[3 * a] - LL.cells[3 * b], dy = LL.cells[3 * a + 1] - LL.cells[3 * b + 1],
                dz = LL.cells[3 * a + 2] - LL.cells[3 * b + 2];
      return (dz + 3) * 49 + (dy + 3) * 7 + (dx + 3);
    };
    auto octant = [&](int q) {
      return (LL.cells[3 * q] & 1) | ((LL.cells[3 * q + 1] & 1) << 1) | ((LL.cells[3 * q + 2] & 1) << 2);
    };
    const long rc2 = (long)rc * rc;
    // Reduced-precision mode: the weights R (R^T R = Z^T Z) come from sums of
    // per-offset Gram matrices of the translation table and an FP64 Cholesky,
    // instead of a QR of the tall stacked table blocks.  Squaring the
    // condition number resolves directions down to ~1e-7 of the largest,
    // below what FP32 recompression distinguishes.
    std::vector<double*> rz_row, rz_col;
    if (prec == P32 && rc <= 128) {
      double* gk = levelmem.alloc((size_t)2 * 343 * rc2);  // K^T K, then K K^T, per offset
      double* gm = levelmem.alloc((size_t)8 * rc2);        // M2M^T M2M per octant
      std::vector<GemmDesc> gg;
      for (int o = 0; o < 343; ++o) {
        const int ox = o % 7 - 3, oy = (o / 7) % 7 - 3, oz = o / 49 - 3;
        if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) continue;
        gg.push_back(gmm(m2l_tab + o * rc2, rc, 1, m2l_tab + o * rc2, rc, 0, gk + o * rc2, rc, rc, rc, rc, 1.0, 0.0));
        gg.push_back(gmm(m2l_tab + o * rc2, rc, 0, m2l_tab + o * rc2, rc, 1, gk + (343 + o) * rc2, rc, rc, rc, rc, 1.0,
                         0.0));
      }
      for (int o = 0; o < 8; ++o)
        gg.push_back(gmm(m2m_tab + o * rc2, rc, 1, m2m_tab + o * rc2, rc, 0, gm + o * rc2, rc, rc, rc, rc, 1.0, 0.0));
      cnt.add_gemm(gg);
      launch_gemm(st, gg, P64);
      std::vector<double*> dst(2 * (size_t)nn);
      std::vector<int> first(2 * (size_t)nn + 1, 0);
      rz_row.resize(nn);
      rz_col.resize(nn);
      double* Rall = scratch().alloc(std::max<size_t>(1, 2 * (size_t)nn * ((rc2 + 31) & ~(size_t)31)));
      for (int q = 0; q < nn; ++q)
        for (int side = 0; side < 2; ++side) {
          const size_t x = 2 * (size_t)q + side;
          double* R = Rall + x * ((rc2 + 31) & ~(size_t)31);
          (side == 0 ? rz_row : rz_col)[q] = R;
          dst[x] = R;
          first[x + 1] = first[x] + (LL.il_ptr[q + 1] - LL.il_ptr[q]) + (kappa > 2 ? 1 : 0);
        }
      std::vector<const double*> terms((size_t)first.back());
      {
        const int nt = host_threads(nn);
        parallel_ranges(nt, [&](int t) {
          const int a0 = (int)((long)nn * t / nt), a1 = (int)((long)nn * (t + 1) / nt);
          for (int q = a0; q < a1; ++q)
            for (int side = 0; side < 2; ++side) {
              size_t y = (size_t)first[2 * (size_t)q + side];
              for (int e = LL.il_ptr[q]; e < LL.il_ptr[q + 1]; ++e) {
                const int l = LL.il[e];
                terms[y++] = side == 0 ? gk + off_index(l, q) * rc2 : gk + (343 + off_index(q, l)) * rc2;
              }
              if (kappa > 2) terms[y++] = gm + octant(q) * rc2;
            }
        });
      }
      launch_gram_sum(st, dst, terms, first, rc);
      launch_chol(st, dst, rc, 1e-13);
    }
    for (int q = 0; q < nn; ++q) {
      Event ev = make_event(W, q);
      ev.r_old = rc;
      ev.n = W.n[q];
      if (!rz_row.empty()) {
        const bool any = (LL.il_ptr[q + 1] > LL.il_ptr[q]) || kappa > 2;
        if (any) {
          ev.z[0].push_back(Blk{rz_row[q], rc, rc, rc, 0});
          ev.z[1].push_back(Blk{rz_col[q], rc, rc, rc, 0});
        }
      } else {
        for (int e = LL.il_ptr[q]; e < LL.il_ptr[q + 1]; ++e) {
          const int l = LL.il[e];
          ev.z[0].push_back(Blk{m2l_tab + off_index(l, q) * rc2, rc, rc, rc, 0});  // K(l,q)
          ev.z[1].push_back(Blk{m2l_tab + off_index(q, l) * rc2, rc, rc, rc, 1});  // K(q,l)^T
        }
        if (kappa > 2) {
          ev.z[0].push_back(Blk{m2m_tab + octant(q) * rc2, rc, rc, rc, 0});  // M2M
          ev.z[1].push_back(Blk{m2m_tab + octant(q) * rc2, rc, rc, rc, 0});  // L2L^T = M2M
        }
      }
      ev.b[0] = Blk{P2M0[q], rc, rc, W.n[q], 0};
      ev.b[1] = Blk{L2P0[q], W.n[q], rc, W.n[q], 1};
      evs.push_back(std::move(ev));
      po.push_back(W.P2M[q]);
      lo.push_back(W.L2P[q]);
      pld.push_back(W.capr[q]);
      lld.push_back(W.n[q]);
    }
    phase("host_init_events", tq);
    in_init = true;
    run_events(evs, W, po, lo, pld, lld, nullptr, 0);
    in_init = false;
    tq = std::chrono::steady_clock::now();
    for (auto& ev : evs) W.r[ev.q] = ev.k;
    // M2L blocks T'_a K T_b; M2M = M2M_tab T; L2L = T' M2M_tab^T
    std::vector<GemmDesc> g1, g2;
    if (rc <= 64) {
      // on the device (k_m2l_init), the entries grouped by offset so that each
      // translation block is staged once per chunk
      std::vector<int> per(344, 0), ent;
      std::vector<int> offs(LL.il.size(), -1);
      for (int a = 0; a < nn; ++a)
        for (int e = LL.il_ptr[a]; e < LL.il_ptr[a + 1]; ++e) {
          const int b = LL.il[e];
          const int ka = evs[a].k, kb = evs[b].k;
          if (!ka || !kb) continue;
          offs[e] = off_index(a, b);
          per[offs[e] + 1]++;
          cnt.gemm += 2.0 * ka * rc * rc + 2.0 * ka * kb * rc;
        }
      for (int o = 0; o < 343; ++o) per[o + 1] += per[o];
      ent.assign(per[343], 0);
      std::vector<int> fill(per.begin(), per.end() - 1);
      for (size_t e = 0; e < offs.size(); ++e)
        if (offs[e] >= 0) ent[fill[offs[e]]++] = (int)e;
      std::vector<M2lChunk> chunks;
      for (int o = 0; o < 343; ++o)
        for (int f = per[o]; f < per[o + 1]; f += 64) chunks.push_back(M2lChunk{o, f, std::min(64, per[o + 1] - f), 0});
      std::vector<int> kv(nn);
      std::vector<const double*> tv(nn), tpv(nn);
      for (int q = 0; q < nn; ++q) {
        kv[q] = evs[q].k;
        tv[q] = evs[q].T;
        tpv[q] = evs[q].Tp;
      }
      const M2lTables mt{st.push(ent), W.d_il_row, W.d_il, W.d_far, W.d_capr, st.push(kv), st.push(tv), st.push(tpv),
                         m2l_tab, rc, 0};
      launch_m2l_init(st, chunks, mt, prec);
    } else {
      std::vector<double*> tmp(LL.il.size());
      for (int a = 0; a < nn; ++a)
        for (int e = LL.il_ptr[a]; e < LL.il_ptr[a + 1]; ++e) {
          const int b = LL.il[e];
          const int ka = evs[a].k, kb = evs[b].k;
          if (!ka || !kb) continue;
          tmp[e] = scratch().alloc((size_t)ka * rc);
          g1.push_back(gmm(evs[a].Tp, ka, 0, m2l_tab + off_index(a, b) * rc2, rc, 0, tmp[e], ka, ka, rc, rc, 1.0, 0.0));
          g2.push_back(gmm(tmp[e], ka, 0, evs[b].T, rc, 0, W.far[e], W.capr[a], ka, kb, rc, 1.0, 0.0));
        }
    }
    if (kappa > 2)
      for (int q = 0; q < nn; ++q) {
        const int k = evs[q].k;
        if (!k) continue;
        g1.push_back(gmm(m2m_tab + octant(q) * rc2, rc, 0, evs[q].T, rc, 0, W.M2M[q], rc, rc, k, rc, 1.0, 0.0));
        g1.push_back(gmm(evs[q].Tp, k, 0, m2m_tab + octant(q) * rc2, rc, 1, W.L2L[q], W.capr[q], k, rc, rc, 1.0, 0.0));
      }
    cnt.add_gemm(g1);
    cnt.add_gemm(g2);
    launch_gemm(st, g1, prec);
    launch_gemm(st, g2, prec);
    phase("host_init_m2l", tq);
  }

  // ------------------------------------------------------------------ one color
  // A color is done in three stages (Algorithm 1 over the color's nodes):
  //   phase A     pivots and Schur complements (launched);
  //   events      recompression of the live neighbours that received far
  //               fill-ins, the ranks read back (the stream is synchronized),
  //               the new bases and transforms (launched);
  //   phase B/C   interaction-list blocks re-expressed in the new bases, fill-in
  //               coefficients added (launched).
  // run() issues them as A(c), B/C(c-1), events(c): the next color's pivots
  // and Schur updates read only near blocks and the just re-based P2M/L2P, never
  // the far blocks that B/C(c-1) rewrite, so the GPU executes them while the
  // host builds B/C(c-1); events(c) read far blocks and come after.
  struct FarFill {
    int a, b;
    const double* Fp;
    int ld, rows, cols;
    int fx;  // position of (a, b) in the IL CSR
  };
  struct ColorState {
    std::vector<int> grp;
    int sel = 0;  // scratch arena
    std::vector<FarFill> fills;
    std::vector<int> slot_of, rebase_order, trigger_of;
    std::vector<std::vector<Blk>> rowfill_v, colfill_v;
    std::vector<Event> evs;
    std::vector<int> r_before;
  };

  void color_phase_a(Work& W, ColorState& cs, LevelFactor& LF) {
    const LevelLists& LL = *W.LL;
    auto tp = std::chrono::steady_clock::now();
    scratch_sel = cs.sel;
    scratch().reset();
    const std::vector<int>& grp = cs.grp;
    const int ng = (int)grp.size();
    if (info_cap < ng) {
      if (d_info) {
        registry().remove_range(d_info, sizeof(int) * info_cap);
        cudaFree(d_info);
      }
      CK(cudaMalloc(&d_info, sizeof(int) * std::max(ng, 64)));
      info_cap = std::max(ng, 64);
      registry().add(d_info, sizeof(int) * info_cap);
    }
    // ---- pivots
    auto& cpi = fresh(L.cpi);
    auto& inv = fresh(L.inv);
    std::vector<double*> Pi(ng);
    for (int g = 0; g < ng; ++g) {
      const int i = grp[g];
      const int ni = W.n[i], ri = W.r[i], m = ni + ri;
      Pi[g] = F.persist.alloc((size_t)std::max(1, m * m));
      if (m == 0) continue;
      cpi.push_back(cpy(W.nb[0][W.slot(i, i)], ni, Pi[g], m, ni, ni));
      if (ri) {
        cpi.push_back(cpy(W.L2P[i], ni, Pi[g] + (long)ni * m, m, ni, ri));
        cpi.push_back(cpy(W.P2M[i], W.capr[i], Pi[g] + ni, m, ri, ni));
        cpi.push_back(cpy(nullptr, 0, Pi[g] + ni + (long)ni * m, m, ri, ri));
      }
      inv.push_back(InvDesc{Pi[g], m, m, d_info + g, 0});
      cnt.inv += 2.0 * ((double)m * m * m);
    }
    CK(cudaMemsetAsync(d_info, 0, sizeof(int) * ng, s));
    launch_copy(st, cpi);
    launch_inv(st, inv);
    phase("host_pivots", tp);
    auto tq = tp;
    // ---- Schur complements of the cliques
    auto& cg = fresh(L.cg);
    auto& sc = fresh(L.sc);
    auto& scat = fresh(L.scat);
    int maxdeg = 0;
    // near-structure state of this color for the scatter kernel (before the
    // color's own nodes count as eliminated; their neighbours are not in it)
    auto& el8 = fresh(L.el8);
    el8.assign(W.elim.begin(), W.elim.end());
    auto& gx = fresh(L.gx);
    auto& gf = fresh(L.gf);
    auto& fills = cs.fills;
    // per-node fill lists, indexed through the order in which nodes first
    // receive a far fill (the re-base order)
    auto& slot_of = cs.slot_of;
    slot_of.assign(W.nn, -1);
    auto& rebase_order = cs.rebase_order;
    auto& rowfill_v = cs.rowfill_v;
    auto& colfill_v = cs.colfill_v;
    auto& trigger_of = cs.trigger_of;
    int cur_i = -1;
    auto rebase_slot = [&](int q) {
      if (slot_of[q] < 0) {
        slot_of[q] = (int)rebase_order.size();
        rebase_order.push_back(q);
        rowfill_v.emplace_back();
        colfill_v.emplace_back();
        trigger_of.push_back(cur_i);
      }
      return slot_of[q];
    };
    // The per-node work runs on host threads over contiguous node ranges.  What
    // each node produces (descriptors, far pairs) is merged afterwards in node
    // order, so launches, re-base order and results are those of a serial loop.
    struct FarRec {
      int q, q2;
      const double* src;
      int M, mq, mq2, fx;
      int g;  // position of the eliminated node in the color
    };
    // scratch of every node (L, U, X, F, Yr), one allocation in node order
    std::vector<double*> nbase(ng, nullptr);
    {
      auto rup = [](size_t x) { return (x + 31) & ~(size_t)31; };  // the arena's 256-byte granules
      std::vector<size_t> offs(ng, 0);
      size_t tot = 0;
      for (int g = 0; g < ng; ++g) {
        const int i = grp[g];
        const int ni = W.n[i], ri = W.r[i], m = ni + ri;
        int M = 0;
        for (int e = LL.nbr_ptr[i]; e < LL.nbr_ptr[i + 1]; ++e) M += W.dim(LL.nbr[e]);
        offs[g] = tot;
        if (M && m)
          tot += rup((size_t)M * std::max(1, ni)) + rup((size_t)std::max(1, ni) * M) + rup((size_t)M * m) +
                 rup((size_t)M * M) + rup((size_t)std::max(1, ri) * M);
      }
      double* blk = tot ? scratch().alloc(tot) : nullptr;
      for (int g = 0; g < ng; ++g) nbase[g] = blk ? blk + offs[g] : nullptr;
    }
    const int nth = host_threads(ng);
    if ((int)W.marks.size() < nth) W.marks.resize(nth);
    for (int t = 0; t < nth; ++t)
      if ((int)W.marks[t].size() != W.nn) W.marks[t].assign(W.nn, -1);
    // each thread fills local lists, handed over once at the end (per-thread
    // slots of shared arrays written on every push would share cache lines)
    std::vector<std::vector<CopyDesc>> cg_t(nth), sc_t(nth);
    std::vector<std::vector<GemmDesc>> gx_t(nth), gf_t(nth);
    std::vector<std::vector<ScatterDesc>> scat_t(nth);
    std::vector<std::vector<FarRec>> far_t(nth);
    std::vector<int> maxdeg_t(nth, 0);
    parallel_ranges(nth, [&](int t) {
      std::vector<int>& mark = W.marks[t];
      std::vector<CopyDesc> cgv, scv;
      std::vector<GemmDesc> gxv, gfv;
      std::vector<ScatterDesc> scatv;
      std::vector<FarRec> farv;
      int maxdeg_l = 0;
      const int g0 = (int)((long)ng * t / nth), g1 = (int)((long)ng * (t + 1) / nth);
      std::vector<int> roff, dims;
      for (int g = g0; g < g1; ++g) {
        const int i = grp[g];
        const int ni = W.n[i], ri = W.r[i], m = ni + ri;
        const int q0 = LL.nbr_ptr[i], q1 = LL.nbr_ptr[i + 1];
        NodeFactor& nf = LF.nf[i];
        nf.piinv = Pi[g];
        nf.n = ni;
        nf.r = ri;
        roff.clear();
        dims.clear();
        int M = 0;
        for (int e = q0; e < q1; ++e) {
          const int q = LL.nbr[e];
          roff.push_back(M);
          dims.push_back(W.dim(q));
          M += W.dim(q);
          nf.nb.push_back(q);
          nf.was_elim.push_back(W.elim[q]);
          const int sq = W.slot(q, i), si = W.slot(i, q);
          nf.lcol.push_back(W.nb[W.elim[q]][sq]);
          nf.lcol_ld.push_back(W.n[q]);
          nf.lcol_rows.push_back(W.dim(q));
          nf.urow.push_back(W.nb[W.elim[q]][si]);
          nf.urow_cols.push_back(W.dim(q));
        }
        // -A22 -> self block of R_i x y_i
        if (ri) scv.push_back(cpy(Pi[g] + ni + (long)ni * m, m, W.nb[2][W.slot(i, i)], ni, ri, ri, -1.0, 0.0));
        if (M == 0 || m == 0) continue;
        auto rup = [](size_t x) { return (x + 31) & ~(size_t)31; };
        double* L = nbase[g];
        double* U = L + rup((size_t)M * std::max(1, ni));
        double* X = U + rup((size_t)std::max(1, ni) * M);
        double* Fm = X + rup((size_t)M * m);
        double* Yr = Fm + rup((size_t)M * M);
        for (size_t a = 0; a < nf.nb.size(); ++a) {
          const int q = nf.nb[a];
          if (ni && dims[a]) {
            cgv.push_back(cpy(nf.lcol[a], W.n[q], L + roff[a], M, dims[a], ni));
            cgv.push_back(cpy(nf.urow[a], ni, U + (long)roff[a] * ni, ni, ni, dims[a]));
          }
        }
        if (ni) {
          gxv.push_back(gmm(L, M, 0, Pi[g], m, 0, X, M, M, m, ni, 1.0, 0.0));  // X = L [A11 A12]
          gfv.push_back(gmm(X, M, 0, U, ni, 0, Fm, M, M, M, ni, -1.0, 0.0));  // F = -X[:, :ni] U
          if (ri) gfv.push_back(gmm(Pi[g] + ni, m, 0, U, ni, 0, Yr, ri, ri, M, ni, 1.0, 0.0));  // A21 U
          scatv.push_back(ScatterDesc{Fm, M, i});
          maxdeg_l = std::max(maxdeg_l, q1 - q0);
        }
        for (size_t a = 0; a < nf.nb.size(); ++a) {
          const int q = nf.nb[a];
          const int mq = dims[a];
          // O(1) slot lookups of q's near blocks in the pair loop below
          mark[q] = W.slot_ptr[q];
          for (int e = LL.nbr_ptr[q]; e < LL.nbr_ptr[q + 1]; ++e) mark[LL.nbr[e]] = W.slot_ptr[q] + 1 + (e - LL.nbr_ptr[q]);
          // row-var(q) x y_i  <- L A12
          if (mq && ri && ni)
            scv.push_back(cpy(X + roff[a] + (long)ni * M, M, W.nb[W.elim[q] + 1][W.slot(q, i)], W.n[q], mq, ri));
          else if (mq && ri)
            scv.push_back(cpy(nullptr, 0, W.nb[W.elim[q] + 1][W.slot(q, i)], W.n[q], mq, ri));
          // R_i x col-var(q)  <- A21 U
          if (mq && ri && ni)
            scv.push_back(cpy(Yr + (long)roff[a] * ri, ri, W.nb[1 + W.elim[q]][W.slot(i, q)], ni, ri, mq));
          else if (mq && ri)
            scv.push_back(cpy(nullptr, 0, W.nb[1 + W.elim[q]][W.slot(i, q)], ni, ri, mq));
          for (size_t b2 = 0; b2 < nf.nb.size(); ++b2) {
            const int q2 = nf.nb[b2];
            const int mq2 = dims[b2];
            if (!mq || !mq2 || !ni) continue;
            if (mark[q2] >= 0) continue;  // near pair: added on the device (k_schur_scatter)
            const int fx = W.farix(q, q2);
            IFMM_REQUIRE(fx >= 0, IFMM_EINVAL, "internal: clique pair neither near nor far");
            farv.push_back(FarRec{q, q2, Fm + roff[a] + (long)roff[b2] * M, M, mq, mq2, fx, g});
          }
          mark[q] = -1;
          for (int e = LL.nbr_ptr[q]; e < LL.nbr_ptr[q + 1]; ++e) mark[LL.nbr[e]] = -1;
        }
      }
      cg_t[t].swap(cgv);
      sc_t[t].swap(scv);
      gx_t[t].swap(gxv);
      gf_t[t].swap(gfv);
      scat_t[t].swap(scatv);
      far_t[t].swap(farv);
      maxdeg_t[t] = maxdeg_l;
    });
    phase("host_schur_nodes", tq);
    for (int t = 0; t < nth; ++t) {
      cg.insert(cg.end(), cg_t[t].begin(), cg_t[t].end());
      sc.insert(sc.end(), sc_t[t].begin(), sc_t[t].end());
      gx.insert(gx.end(), gx_t[t].begin(), gx_t[t].end());
      gf.insert(gf.end(), gf_t[t].begin(), gf_t[t].end());
      scat.insert(scat.end(), scat_t[t].begin(), scat_t[t].end());
      maxdeg = std::max(maxdeg, maxdeg_t[t]);
    }
    // Far pairs in node order (the threads' node ranges are contiguous and in
    // order, so the threads' lists one after another are that order): the
    // fill-in list; the re-base order (first appearance of a node not yet
    // eliminated, its column role before its row role); and each re-based
    // node's column and row fill lists, in the same order.
    std::vector<size_t> foff(nth + 1, 0);
    for (int t = 0; t < nth; ++t) foff[t + 1] = foff[t] + far_t[t].size();
    for (int t = 0; t < nth; ++t)
      for (const FarRec& f : far_t[t]) {
        cur_i = grp[f.g];
        if (!W.elim[f.q]) rebase_slot(f.q);
        if (!W.elim[f.q2]) rebase_slot(f.q2);
      }
    const int nsl = (int)rebase_order.size();
    fills.resize(foff[nth]);
    // per thread and slot: how many column / row fills; then, after the
    // exclusive prefix over the threads, where the thread's next one goes
    std::vector<std::vector<int>> cpos(nth), rpos(nth);
    parallel_ranges(nth, [&](int t) {
      std::vector<int> cn(nsl, 0), rn(nsl, 0);
      size_t x = foff[t];
      for (const FarRec& f : far_t[t]) {
        fills[x++] = FarFill{f.q, f.q2, f.src, f.M, f.mq, f.mq2, f.fx};
        if (!W.elim[f.q]) ++cn[slot_of[f.q]];
        if (!W.elim[f.q2]) ++rn[slot_of[f.q2]];
      }
      cpos[t].swap(cn);
      rpos[t].swap(rn);
    });
    {
      const int ns = host_threads(nsl);
      parallel_ranges(ns, [&](int u) {
        const int s0 = (int)((long)nsl * u / ns), s1 = (int)((long)nsl * (u + 1) / ns);
        for (int sl = s0; sl < s1; ++sl) {
          int c = 0, r = 0;
          for (int t = 0; t < nth; ++t) {
            const int a = cpos[t][sl], b = rpos[t][sl];
            cpos[t][sl] = c;
            rpos[t][sl] = r;
            c += a;
            r += b;
          }
          colfill_v[sl].resize(c);
          rowfill_v[sl].resize(r);
        }
      });
    }
    parallel_ranges(nth, [&](int t) {
      std::vector<int>& cp = cpos[t];
      std::vector<int>& rp = rpos[t];
      for (const FarRec& f : far_t[t]) {
        if (!W.elim[f.q]) {
          const int sl = slot_of[f.q];
          colfill_v[sl][cp[sl]++] = Blk{f.src, f.M, f.mq2, W.n[f.q], 1};
        }
        if (!W.elim[f.q2]) {
          const int sl = slot_of[f.q2];
          rowfill_v[sl][rp[sl]++] = Blk{f.src, f.M, f.mq, W.n[f.q2], 0};
        }
      }
    });
    for (int g = 0; g < ng; ++g) W.elim[grp[g]] = 1;
    phase("host_schur_merge", tq);
    launch_copy(st, cg);
    cnt.add_gemm(gx);
    cnt.add_gemm(gf);
    launch_gemm(st, gx, gprec);
    launch_gemm(st, gf, gprec);
    launch_copy(st, sc);
    if (!scat.empty()) {
      const ScatterTables tt{W.d_nbr_ptr, W.d_nbr, W.d_slot_ptr, W.d_n, st.push(W.r), st.push(el8),
                             W.d_nb[0], W.d_nb[1], W.d_nb[2]};
      launch_schur_scatter(st, scat, tt, maxdeg);
    }
    phase("host_schur_launch", tq);
    phase("host_schur", tp);
  }

  void color_events(Work& W, ColorState& cs) {
    const LevelLists& LL = *W.LL;
    auto tp = std::chrono::steady_clock::now();
    scratch_sel = cs.sel;
    const int ng = (int)cs.grp.size();
    auto& slot_of = cs.slot_of;
    auto& rowfill_v = cs.rowfill_v;
    auto& colfill_v = cs.colfill_v;
    auto& trigger_of = cs.trigger_of;
    // ---- recompression events (snapshots: nothing below reads what phase A changes)
    auto& evs = cs.evs;
    std::vector<double*> po, lo;
    std::vector<int> pld, lld;
    cs.r_before = W.r;
    // one event per re-based node, in the re-base order (the nodes are
    // distinct, so the threads touch distinct event counters)
    const int nev = (int)cs.rebase_order.size();
    evs.resize(nev);
    po.resize(nev);
    lo.resize(nev);
    pld.resize(nev);
    lld.resize(nev);
    const int nthe = host_threads(nev);
    parallel_ranges(nthe, [&](int t) {
      const int x0 = (int)((long)nev * t / nthe), x1 = (int)((long)nev * (t + 1) / nthe);
      for (int x = x0; x < x1; ++x) {
        const int q = cs.rebase_order[x];
        Event ev = make_event(W, q, trigger_of[slot_of[q]]);
        ev.r_old = W.r[q];
        ev.n = W.n[q];
        const int rq = W.r[q];
        // weight stacks [M2L_lq (l in IL_q); M2M_q] and [M2L_ql^T; L2L_q^T],
        // gathered on the device (k_zgather): only their height is needed here
        int mzd = 0;
        if (rq) {
          for (int e = LL.il_ptr[q]; e < LL.il_ptr[q + 1]; ++e) mzd += W.r[LL.il[e]];
          if (W.kappa > 2) mzd += rc;
        }
        ev.zq = q;
        ev.mzd = mzd;
        ev.b[0] = Blk{W.P2M[q], W.capr[q], rq, W.n[q], 0};
        ev.b[1] = Blk{W.L2P[q], W.n[q], rq, W.n[q], 1};
        ev.f[0] = std::move(rowfill_v[slot_of[q]]);
        ev.f[1] = std::move(colfill_v[slot_of[q]]);
        evs[x] = std::move(ev);
        po[x] = W.P2M[q];
        lo[x] = W.L2P[q];
        pld[x] = W.capr[q];
        lld[x] = W.n[q];
      }
    });
    phase("host_events", tp);
    const double w0 = t_wait;
    const ZTables zt{W.d_il_ptr, W.d_il, W.d_il_T, W.d_far, W.d_capr, st.push(W.r), W.d_M2M, W.d_L2L, rc,
                     W.kappa > 2 ? 1 : 0};
    run_events(evs, W, po, lo, pld, lld, nullptr, ng, &zt);
    F.stat_add("host_run_events_wait", t_wait - w0);
    phase("host_run_events", tp);
    for (auto& ev : evs) W.r[ev.q] = ev.k;
  }

  void color_phase_bc(Work& W, ColorState& cs) {
    const LevelLists& LL = *W.LL;
    auto tp = std::chrono::steady_clock::now();
    auto tq = tp;
    scratch_sel = cs.sel;
    auto& evs = cs.evs;
    auto& fills = cs.fills;
    const std::vector<int>& r_before = cs.r_before;
    // ---- phase B: re-express blocks that touch a re-based node
    std::vector<int> newk(W.nn, -1);
    std::vector<const Event*> evof(W.nn, nullptr);
    for (auto& ev : evs) {
      newk[ev.q] = ev.k;
      evof[ev.q] = &ev;
    }
    auto& b1 = fresh(L.b1);
    auto& b2 = fresh(L.b2);
    auto& bc1 = fresh(L.bc1);
    auto& bc2 = fresh(L.bc2);
    // M2M and L2L of the re-based nodes: two GEMMs and two copies per event,
    // through temporaries carved in event order from one allocation (256-byte
    // granules, as the arena's own); written by host threads
    if (W.kappa > 2) {
      auto rup = [](size_t x) { return (x + 31) & ~(size_t)31; };
      const int ne = (int)evs.size();
      std::vector<int> slot(ne, -1);
      std::vector<size_t> toff(ne, 0);
      int nq = 0;
      size_t tot = 0;
      for (int x = 0; x < ne; ++x)
        if (evs[x].k && evs[x].r_old) {
          slot[x] = nq++;
          toff[x] = tot;
          tot += 2 * rup((size_t)rc * evs[x].k);
        }
      double* tb = tot ? scratch().alloc(tot) : nullptr;
      b1.resize(2 * (size_t)nq);
      bc1.resize(2 * (size_t)nq);
      const int nthm = host_threads(ne);
      parallel_ranges(nthm, [&](int t) {
        const int x0 = (int)((long)ne * t / nthm), x1 = (int)((long)ne * (t + 1) / nthm);
        for (int x = x0; x < x1; ++x) {
          if (slot[x] < 0) continue;
          const Event& ev = evs[x];
          const int q = ev.q;
          const size_t j = 2 * (size_t)slot[x];
          double* t1 = tb + toff[x];
          double* t2 = t1 + rup((size_t)rc * ev.k);
          registry().add(t1, sizeof(double) * (size_t)rc * ev.k);  // bounds of the pieces (IFMM_CHECK)
          registry().add(t2, sizeof(double) * (size_t)rc * ev.k);
          b1[j] = gmm(W.M2M[q], rc, 0, ev.T, ev.r_old, 0, t1, rc, rc, ev.k, ev.r_old, 1.0, 0.0);
          b1[j + 1] = gmm(ev.Tp, ev.k, 0, W.L2L[q], W.capr[q], 0, t2, ev.k, ev.k, rc, ev.r_old, 1.0, 0.0);
          bc1[j] = cpy(t1, rc, W.M2M[q], rc, rc, ev.k);
          bc1[j + 1] = cpy(t2, ev.k, W.L2L[q], W.capr[q], ev.k, rc);
        }
      });
    }
    // IL entries with an endpoint re-based in this color, each once: an event of
    // node q takes its row entries (q, l), and the transposes (l, q) whose other
    // end l is not re-based (else l's event takes them).  Entries whose ranks
    // all fit the fused kernel's tiles go to one launch; the rest (a rank above
    // 64) keep per-block GEMM descriptors.  The events are split over host
    // threads; the lists are joined in event order.
    const int nev = (int)evs.size();
    const int nthb = host_threads(nev);
    std::vector<std::vector<int>> fast_t(nthb), slow_t(nthb);
    std::vector<int> md_t(nthb, 1);
    std::vector<double> fl_t(nthb, 0.0);
    parallel_ranges(nthb, [&](int t) {
      const int e0 = (int)((long)nev * t / nthb), e1 = (int)((long)nev * (t + 1) / nthb);
      // accumulated in locals: per-thread slots of shared arrays written on
      // every entry would share cache lines between the threads
      std::vector<int> fast_l, slow_l;
      int md_l = 1;
      double fl_l = 0.0;
      size_t bound = 0;
      for (int x = e0; x < e1; ++x) bound += 2 * (size_t)(LL.il_ptr[evs[x].q + 1] - LL.il_ptr[evs[x].q]);
      fast_l.reserve(bound);
      auto take = [&](int e) {
        const int a = W.il_row[e];
        const int b = LL.il[e];
        const int ra = r_before[a], rb = r_before[b];
        const int ka = newk[a] >= 0 ? newk[a] : ra, kb = newk[b] >= 0 ? newk[b] : rb;
        if (!ka || !kb) return;
        const int mx = std::max(std::max(ra, rb), std::max(ka, kb));
        if (mx <= 64) {
          fast_l.push_back(e);
          md_l = std::max(md_l, mx);
          if (ra && rb)
            fl_l += 2.0 * ((newk[a] >= 0 ? (double)ka * rb * ra : 0.0) + (newk[b] >= 0 ? (double)ka * kb * rb : 0.0));
        } else {
          slow_l.push_back(e);
        }
      };
      for (int x = e0; x < e1; ++x) {
        const int q = evs[x].q;
        for (int e = LL.il_ptr[q]; e < LL.il_ptr[q + 1]; ++e) {
          take(e);
          if (newk[LL.il[e]] < 0) take(W.il_T[e]);
        }
      }
      fast_t[t].swap(fast_l);
      slow_t[t].swap(slow_l);
      md_t[t] = md_l;
      fl_t[t] = fl_l;
    });
    phase("host_b_scan", tq);
    auto& fast = fresh(L.tlf);
    int md = 1;
    for (int t = 0; t < nthb; ++t) {
      fast.insert(fast.end(), fast_t[t].begin(), fast_t[t].end());
      md = std::max(md, md_t[t]);
      cnt.gemm += fl_t[t];
    }
    for (int t = 0; t < nthb; ++t)
      for (const int e : slow_t[t]) {
        const int a = W.il_row[e];
        const int b = LL.il[e];
        const int ra = r_before[a], rb = r_before[b];
        const int ka = newk[a] >= 0 ? newk[a] : ra, kb = newk[b] >= 0 ? newk[b] : rb;
        double* t1 = scratch().alloc((size_t)ka * std::max(1, rb));
        if (!ra || !rb) {
          bc2.push_back(cpy(nullptr, 0, W.far[e], W.capr[a], ka, kb));
          continue;
        }
        if (newk[a] >= 0)
          b1.push_back(gmm(evof[a]->Tp, ka, 0, W.far[e], W.capr[a], 0, t1, ka, ka, rb, ra, 1.0, 0.0));
        else
          bc1.push_back(cpy(W.far[e], W.capr[a], t1, ka, ka, rb));
        if (newk[b] >= 0)
          b2.push_back(gmm(t1, ka, 0, evof[b]->T, rb, 0, W.far[e], W.capr[a], ka, kb, rb, 1.0, 0.0));
        else
          bc2.push_back(cpy(t1, ka, W.far[e], W.capr[a], ka, kb));
      }
    cnt.add_gemm(b1);
    cnt.add_gemm(b2);
    launch_gemm(st, b1, prec);
    launch_copy(st, bc1);
    launch_gemm(st, b2, prec);
    launch_copy(st, bc2);
    if (!fast.empty()) {
      auto& tn = fresh(L.tn);
      auto& tpn = fresh(L.tpn);
      tn.assign(W.nn, nullptr);
      tpn.assign(W.nn, nullptr);
      for (auto& ev : evs) {
        tn[ev.q] = ev.T;
        tpn[ev.q] = ev.Tp;
      }
      IlTables t{W.d_il_row, W.d_il, W.d_far, W.d_capr, st.push(r_before), st.push(newk), st.push(tn), st.push(tpn)};
      launch_il_transform(st, fast, t, md, prec);
    }
    phase("host_b_launch", tq);
    phase("host_phase_b", tp);
    // ---- phase C: fill-in coefficients in the new bases
    auto& c1 = fresh(L.c1);
    auto& c2 = fresh(L.c2);
    auto& cc = fresh(L.cc);
    // The fills are split over host threads and the lists joined in fill
    // order.  The temporaries of fills with both ends re-based come from one
    // allocation, carved in fill order into the arena's 256-byte granules.
    const int nfill = (int)fills.size();
    const int nthc = host_threads(nfill);
    auto rup = [](size_t x) { return (x + 31) & ~(size_t)31; };
    auto both_live = [&](const FarFill& f) { return newk[f.a] >= 0 && newk[f.b] >= 0 && W.r[f.a] && W.r[f.b]; };
    std::vector<size_t> toff(nthc + 1, 0);
    parallel_ranges(nthc, [&](int t) {
      const int f0 = (int)((long)nfill * t / nthc), f1 = (int)((long)nfill * (t + 1) / nthc);
      size_t z = 0;
      for (int x = f0; x < f1; ++x)
        if (both_live(fills[x])) z += rup((size_t)W.r[fills[x].a] * fills[x].cols);
      toff[t + 1] = z;
    });
    for (int t = 0; t < nthc; ++t) toff[t + 1] += toff[t];
    double* tbase = toff[nthc] ? scratch().alloc(toff[nthc]) : nullptr;
    std::vector<std::vector<GemmDesc>> c1_t(nthc), c2_t(nthc);
    std::vector<std::vector<CopyDesc>> cc_t(nthc);
    parallel_ranges(nthc, [&](int t) {
      const int f0 = (int)((long)nfill * t / nthc), f1 = (int)((long)nfill * (t + 1) / nthc);
      std::vector<GemmDesc> c1l, c2l;
      std::vector<CopyDesc> ccl;
      c2l.reserve(f1 - f0);
      double* tnext = tbase ? tbase + toff[t] : nullptr;
      for (int x = f0; x < f1; ++x) {
        const FarFill& f = fills[x];
        const int a = f.a, b = f.b;
        const bool la = newk[a] >= 0, lb = newk[b] >= 0;  // live (re-based this color)
        const int ka = W.r[a], kb = W.r[b];
        double* dst = W.far[f.fx];
        const int ldd = W.capr[a];
        if (!ka || !kb) continue;
        if (la && lb) {
          double* tt = tnext;
          tnext += rup((size_t)ka * f.cols);
          registry().add(tt, sizeof(double) * (size_t)ka * f.cols);  // bounds of the piece (IFMM_CHECK)
          c1l.push_back(gmm(W.L2P[a], W.n[a], 1, f.Fp, f.ld, 0, tt, ka, ka, f.cols, f.rows, 1.0, 0.0));
          c2l.push_back(gmm(tt, ka, 0, W.P2M[b], W.capr[b], 1, dst, ldd, ka, kb, f.cols, 1.0, 1.0));
        } else if (la) {
          c2l.push_back(gmm(W.L2P[a], W.n[a], 1, f.Fp, f.ld, 0, dst, ldd, ka, kb, f.rows, 1.0, 1.0));
        } else if (lb) {
          c2l.push_back(gmm(f.Fp, f.ld, 0, W.P2M[b], W.capr[b], 1, dst, ldd, ka, kb, f.cols, 1.0, 1.0));
        } else {
          ccl.push_back(cpy(f.Fp, f.ld, dst, ldd, ka, kb, 1.0, 1.0));
        }
      }
      c1_t[t].swap(c1l);
      c2_t[t].swap(c2l);
      cc_t[t].swap(ccl);
    });
    for (int t = 0; t < nthc; ++t) {
      c1.insert(c1.end(), c1_t[t].begin(), c1_t[t].end());
      c2.insert(c2.end(), c2_t[t].begin(), c2_t[t].end());
      cc.insert(cc.end(), cc_t[t].begin(), cc_t[t].end());
    }
    phase("host_c_loop", tq);
    cnt.add_gemm(c1);
    cnt.add_gemm(c2);
    launch_gemm(st, c1, prec);
    launch_gemm(st, c2, prec);
    launch_copy(st, cc);
    phase("host_c_launch", tq);
    phase("host_phase_c", tp);
  }

  // ------------------------------------------------------------------ top level
  void top(Work& W) {
    const LevelLists& LL = *W.LL;
    F.top_off.assign(W.nn + 1, 0);
    for (int a = 0; a < W.nn; ++a) F.top_off[a + 1] = F.top_off[a] + W.r[a];
    const int nt = F.top_off[W.nn];
    F.ntop = nt;
    F.top_inv = F.persist.alloc((size_t)std::max(1, nt) * std::max(1, nt));
    if (!nt) return;
    std::vector<CopyDesc> cc;
    for (int a = 0; a < W.nn; ++a)
      for (int b = 0; b < W.nn; ++b) {
        if (!W.r[a] || !W.r[b]) continue;
        const int sl = W.slot(a, b);
        double* dst = F.top_inv + F.top_off[a] + (long)F.top_off[b] * nt;
        if (sl >= 0) {
          cc.push_back(cpy(W.nb[2][sl], W.n[a], dst, nt, W.r[a], W.r[b]));
        } else {
          const int fx = W.farix(a, b);
          IFMM_REQUIRE(fx >= 0, IFMM_EINVAL, "internal: level-2 pair neither near nor far");
          cc.push_back(cpy(W.far[fx], W.capr[a], dst, nt, W.r[a], W.r[b]));
        }
      }
    (void)LL;
    launch_copy(st, cc);
    double* wk = scratch().alloc(2 * (size_t)nt);
    int* wi = (int*)scratch().alloc((size_t)nt);
    int* info = (int*)scratch().alloc(1);
    big_inverse(s, F.top_inv, nt, nt, wi, wk, info);
    cnt.lu += 2.0 * std::pow((double)nt, 3);
    int hinfo = 0;
    CK(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st.reset();
    IFMM_REQUIRE(hinfo == 0, IFMM_ESINGULAR, "singular top-level system");
  }

  void run() {
    const int ell = T.depth;
    F.lv.assign(ell + 1, LevelFactor());
    m2m_tab = F.persist.alloc((size_t)8 * rc * rc);
    launch_m2m_table(s, m2m_tab, p, kernel_dof(F.k));
    std::unique_ptr<Work> prev;
    auto t0 = std::chrono::steady_clock::now();
    for (int kappa = ell; kappa >= 2; --kappa) {
      auto tl = std::chrono::steady_clock::now();
      std::unique_ptr<Work> W(new Work());
      // the child level's blocks stay alive until this level's initial copies ran
      DeviceArena child_mem;
      child_mem.swap(levelmem);
      prof_level_tag() = kappa;
      cur_level = kappa;
      auto ti = std::chrono::steady_clock::now();
      init_level(*W, kappa, prev.get());
      phase("host_init", ti);
      wait();
      phase("host_init_wait", ti);
      st.reset();
      child_mem.release();
      prev.reset();
      LevelFactor& LF = F.lv[kappa];
      LF.kappa = kappa;
      LF.nn = W->nn;
      LF.nf.assign(W->nn, NodeFactor());
      LF.n = W->n;
      const LevelLists& LL = T.lv[kappa];
      std::unique_ptr<ColorState> pend;  // the previous color, its phase B/C not yet issued
      for (size_t c = 0; c + 1 < LL.group_ptr.size(); ++c) {
        std::unique_ptr<ColorState> cs(new ColorState());
        cs->grp.assign(LL.group.begin() + LL.group_ptr[c], LL.group.begin() + LL.group_ptr[c + 1]);
        cs->sel = (int)(c & 1);
        color_phase_a(*W, *cs, LF);
        if (pend) color_phase_bc(*W, *pend);
        color_events(*W, *cs);
        LF.order.push_back(cs->grp);
        pend = std::move(cs);
      }
      if (pend) color_phase_bc(*W, *pend);
      pend.reset();
      LF.r = W->r;
      if (kappa == 2) top(*W);
      wait();
      st.reset();
      auto te = std::chrono::steady_clock::now();
      F.stat("time_level_" + std::to_string(kappa), std::chrono::duration<double>(te - tl).count());
      prev = std::move(W);
    }
    prof_level_tag() = -1;
    build_solve_plan(F, s);
    CK(cudaStreamSynchronize(s));
    levelmem.release();
    scratch_buf[0].release();
    scratch_buf[1].release();
    // the solve reads its own packed copies: the factor's block pool goes
    F.stat("bytes_factor", (double)F.persist.high);
    F.persist.release();
    for (auto& LF : F.lv)
      for (auto& nf : LF.nf) {
        nf.piinv = nullptr;
        nf.lcol.clear();
        nf.urow.clear();
      }
    F.top_inv = nullptr;
    auto t1 = std::chrono::steady_clock::now();
    F.stat("time_factor", std::chrono::duration<double>(t1 - t0).count());
    F.stat("flops_gemm", cnt.gemm);
    F.stat("flops_inv", cnt.inv);
    F.stat("flops_qr", cnt.qr);
    F.stat("flops_svd", cnt.svd);
    F.stat("flops_lu", cnt.lu);
    F.stat("flops_total", cnt.total());
    F.stat("time_device_wait", t_wait);
    F.stat("learned_events", n_learned);
    F.stat("learned_sketched", n_capped);
    F.stat("learned_fallbacks", n_fallback);
    F.stat("qrcp_steps", qrcp_steps);
  }

  ~Factorizer() {
    if (d_mlp) cudaFree(d_mlp);
    if (d_info) {
      registry().remove_range(d_info, sizeof(int) * info_cap);
      cudaFree(d_info);
    }
  }
};

}  // namespace ifmm

using namespace ifmm;

ifmm_fact::~ifmm_fact() {
  if (plan.graph) cudaGraphExecDestroy(plan.graph);
  if (plan.graph_def) cudaGraphDestroy(plan.graph_def);
}

extern "C" {

ifmm_status ifmm_factor(const ifmm_tree* t, const ifmm_kernel* k, const ifmm_opts* o, void* stream,
                        ifmm_fact** out) {
  if (out) *out = nullptr;
  ifmm_fact* F = nullptr;
  try {
    IFMM_REQUIRE(t && k && o && out, IFMM_EINVAL, "NULL argument");
    IFMM_REQUIRE(t->sigma >= 3, IFMM_EINVAL, "call ifmm_color before ifmm_factor");
    IFMM_REQUIRE(o->cheb_order >= 2 && o->cheb_order <= 6, IFMM_EINVAL, "cheb_order must be in [2, 6]");
    IFMM_REQUIRE(o->eps >= 0.0 && o->eps < 1.0, IFMM_EINVAL, "eps must be in [0, 1)");
    IFMM_REQUIRE(o->rank_mode >= 0 && o->rank_mode <= 2, IFMM_EINVAL, "bad rank_mode");
    IFMM_REQUIRE(o->precision >= 0 && o->precision <= 2, IFMM_EINVAL, "bad precision");
    const_cast<ifmm_tree*>(t)->ensure_device();
    F = new ifmm_fact();
    F->t = t;
    F->k = *k;
    F->o = *o;
    F->p = o->cheb_order;
    F->rc = kernel_dof(*k) * o->cheb_order * o->cheb_order * o->cheb_order;
    IFMM_REQUIRE(k->wavenumber == 0.0 || k->arith == IFMM_ARITH_FP64, IFMM_EINVAL,
                 "the Helmholtz kernel takes the FP64 direct-sum matvec (arith IFMM_ARITH_FP64)");
    {
      Factorizer fz(*F, (cudaStream_t)stream);
      fz.run();
    }
    F->o.replay = nullptr;  // the caller's table is not kept
    F->o.mlp = nullptr;
    *out = F;
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    delete F;
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    delete F;
    return IFMM_ENOMEM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    delete F;
    return IFMM_ECUDA;
  }
}

void ifmm_fact_free(ifmm_fact* f) { delete f; }

ifmm_status ifmm_fact_ranks(const ifmm_fact* f, int32_t* buf, int64_t cap, int64_t* count) {
  if (!f || !count) {
    set_last_error("NULL argument");
    return IFMM_EINVAL;
  }
  *count = (int64_t)f->rank_log.size() * 4;
  for (int64_t e = 0; e < *count && e < cap && buf; ++e) buf[e] = f->rank_log[e / 4][e % 4];
  return IFMM_OK;
}

ifmm_status ifmm_fact_events(const ifmm_fact* f, float* features, int32_t* ranks, int64_t cap, int64_t* count) {
  if (!f || !count) {
    set_last_error("NULL argument");
    return IFMM_EINVAL;
  }
  *count = (int64_t)f->rank_log.size();
  for (int64_t e = 0; e < *count && e < cap; ++e) {
    if (features) memcpy(features + e * IFMM_MLP_IN, &f->event_feat[e * IFMM_MLP_IN], sizeof(float) * IFMM_MLP_IN);
    if (ranks) ranks[e] = f->rank_log[e][3];
  }
  return IFMM_OK;
}

ifmm_status ifmm_fact_stats(const ifmm_fact* f, double* buf, int64_t cap, int64_t* count) {
  if (!f || !count) {
    set_last_error("NULL argument");
    return IFMM_EINVAL;
  }
  *count = (int64_t)f->stats.size();
  for (int64_t e = 0; e < *count && e < cap && buf; ++e) buf[e] = f->stats[e].second;
  return IFMM_OK;
}

const char* ifmm_fact_stat_name(const ifmm_fact* f, int64_t index) {
  if (!f || index < 0 || index >= (int64_t)f->stats.size()) return nullptr;
  return f->stats[index].first.c_str();
}

}  // extern "C"
