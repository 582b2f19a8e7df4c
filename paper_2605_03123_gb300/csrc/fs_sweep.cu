// Givens-rotation sweeps and per-configuration phases.
//
// An orbital rotation of one spin acts on every "vector" of the state that
// holds all strings of that spin: the columns for alpha (dir 0), the rows
// for beta (dir 1).  A slab of KV such vectors is staged in shared memory
// (split over a thread-block cluster when one vector exceeds one SM's shared
// memory), every Givens rotation of the program is applied to it in order
// (§3.2.3: each rotation updates the amplitude pairs (I, I^{p->p+1})), and
// the slab is written back once, multiplied by the configuration phases
// (the diagonal layer of the decomposition, and optionally a fused
// diagonal-Coulomb / number-operator evolution, §3.2.1-§3.2.2).
#include "fs_sweep_kern.cuh"

namespace fs {

// Instantiated in fs_sweep_f32fwd.cu, fs_sweep_f32rev.cu, fs_sweep_f32batch.cu.
extern template void dispatch_cs<float, 1, false, 6, 256, WProg<float>, false>(
    int, const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
extern template void dispatch_cs<float, 1, false, 6, 512, WProg<float>, false>(
    int, const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
extern template void launch_sweep_t<float, 1, 1, false, 6, 256, false, WProg<float>, false, true>(
    const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
extern template void launch_sweep_t<float, 1, 1, false, 6, 512, false, WProg<float>, false, true>(
    const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
extern template void launch_sweep_t<float, 1, 2, true, 6, 512, false, WProg<float>, false, true>(
    const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
extern template void dispatch_cs<float, 2, true, 5, 512, WProg<float>, false>(
    int, const SweepGeom&, const WProg<float>&, const Mat&, int, size_t, cudaStream_t);
extern template void launch_batch_t<float, 1, false, 6, 256, false>(const SweepJob*, int, int, int*,
                                                                   size_t, int, cudaStream_t);
extern template void launch_batch_t<float, 1, false, 6, 512, false>(const SweepJob*, int, int, int*,
                                                                   size_t, int, cudaStream_t);
extern template void launch_batch_t<float, 1, false, 6, 256, false, true>(const SweepJob*, int, int, int*,
                                                                         size_t, int, cudaStream_t);
extern template void launch_batch_t<float, 1, false, 6, 512, false, true>(const SweepJob*, int, int, int*,
                                                                         size_t, int, cudaStream_t);
extern template void launch_batch_t<float, 2, true, 6, 512, false, true>(const SweepJob*, int, int, int*,
                                                                 size_t, int, cudaStream_t);

// The B images of the tensor-core steps of one program, FP64 on the device:
// per step, V = G_k ... G_1 (the step's Givens rotations in the window's
// local orbitals, applied first to last), then for each class m the
// compound matrix C_m(V)[S', S] = det V[S', S] in its real form
// [[Re, -Im], [Im, Re]] (rows n = output reals, columns k = input reals,
// re/im interleaved), split into three BF16 pieces (each the nearest BF16
// of the remainder so far), K-major core matrices (see tc::b_offset).  One
// block per step.
__global__ void __launch_bounds__(256)
    k_tc_bmats(const __grid_constant__ WProg<double> p, unsigned char* out) {
  __shared__ double2 V[tc::kW * tc::kW];
  const int st = blockIdx.x;
  unsigned char* img = out + (size_t)st * tc::kStepBytes;
  for (int i = threadIdx.x; i < tc::kStepBytes / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(img)[i] = 0u;
  if (threadIdx.x == 0) {
    for (int i = 0; i < tc::kW; ++i)
      for (int j = 0; j < tc::kW; ++j) V[i * tc::kW + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    for (int q = p.g0[st]; q < p.g0[st + 1]; ++q) {
      const int u = p.u[q];
      const double c = p.c[q], sr = p.sr[q], si = p.si[q];
      for (int j = 0; j < tc::kW; ++j) {
        const double2 x = V[u * tc::kW + j], y = V[(u + 1) * tc::kW + j];
        // row u <- c x + s y, row u+1 <- -conj(s) x + c y
        V[u * tc::kW + j] = make_double2(c * x.x + sr * y.x - si * y.y, c * x.y + sr * y.y + si * y.x);
        V[(u + 1) * tc::kW + j] =
            make_double2(-(sr * x.x + si * x.y) + c * y.x, -(sr * x.y - si * x.x) + c * y.y);
      }
    }
  }
  __syncthreads();
  for (int m = 1; m < tc::kW; ++m) {
    const int ns = tc::binom6(m), kpad = tc::kp(m);
    for (int idx = threadIdx.x; idx < ns * ns; idx += blockDim.x) {
      const int ip = idx / ns, iq = idx - ip * ns;
      const int rm = win_mask(tc::kW, m, ip), cm = win_mask(tc::kW, m, iq);
      double2 a[5 * 5];
      int r = 0;
      for (int i = 0; i < tc::kW; ++i) {
        if (!((rm >> i) & 1)) continue;
        int cc = 0;
        for (int j = 0; j < tc::kW; ++j)
          if ((cm >> j) & 1) a[r * m + (cc++)] = V[i * tc::kW + j];
        ++r;
      }
      // det by Gaussian elimination with partial pivoting
      double dr = 1, di = 0;
      for (int k = 0; k < m; ++k) {
        int piv = k;
        double best = hypot(a[k * m + k].x, a[k * m + k].y);
        for (int i = k + 1; i < m; ++i) {
          const double h = hypot(a[i * m + k].x, a[i * m + k].y);
          if (h > best) {
            best = h;
            piv = i;
          }
        }
        if (best == 0) {
          dr = di = 0;
          break;
        }
        if (piv != k) {
          for (int j = 0; j < m; ++j) {
            const double2 tmp = a[k * m + j];
            a[k * m + j] = a[piv * m + j];
            a[piv * m + j] = tmp;
          }
          dr = -dr;
          di = -di;
        }
        const double2 pk = a[k * m + k];
        const double nr = dr * pk.x - di * pk.y;
        di = dr * pk.y + di * pk.x;
        dr = nr;
        const double inv = 1.0 / (pk.x * pk.x + pk.y * pk.y);
        for (int i = k + 1; i < m; ++i) {
          const double2 x = a[i * m + k];
          const double fr = (x.x * pk.x + x.y * pk.y) * inv, fi = (x.y * pk.x - x.x * pk.y) * inv;
          for (int j = k + 1; j < m; ++j) {
            const double2 y = a[k * m + j];
            a[i * m + j].x -= fr * y.x - fi * y.y;
            a[i * m + j].y -= fr * y.y + fi * y.x;
          }
        }
      }
      const double ent[4] = {dr, -di, di, dr};  // (2ip, 2iq), (2ip, 2iq+1), (2ip+1, 2iq), (2ip+1, 2iq+1)
      for (int e = 0; e < 4; ++e) {
        const int n = 2 * ip + (e >> 1), k = 2 * iq + (e & 1);
        const int off = tc::b_offset(n, k, kpad);
        double r = ent[e];
        for (int pc = 0; pc < tc::kPieces; ++pc) {  // nearest BF16 of the remainder
          const __nv_bfloat16 b = __float2bfloat16_rn((float)r);
          *reinterpret_cast<__nv_bfloat16*>(img + tc::class_offset(m) + pc * tc::piece_bytes(m) + off) = b;
          r -= (double)__bfloat162float(b);
        }
      }
    }
  }
}

// Transition-reduction passes of a space (built once, on the host; see
// tpass_tables_host).
static void build_tpass_tables(Space* sp) {
  if (sp->tbuilt) return;
  std::vector<TPass>& passes = sp->tpass_h;
  std::vector<TRecord>& recs = sp->trec_h;
  tpass_tables_host(sp->norb, sp->nocc, passes, recs, sp->rkey_h);
  std::vector<TPassDev> pd(passes.size());
  for (size_t i = 0; i < passes.size(); ++i) {
    for (int j = 0; j < 4; ++j) pd[i].q[j] = passes[i].q[j];
    pd[i].keep = passes[i].keep;
    pd[i].rec0 = passes[i].rec0;
    pd[i].rec1 = passes[i].rec1;
    const uint32_t diag = 0x8421u, all = 0xFFFFu;
    pd[i].mode = passes[i].keep == all ? 2 : passes[i].keep == (all & ~diag) ? 1 : 0;
  }
  if (!pd.empty()) {
    FS_CUDA(cudaMalloc(&sp->tpass, pd.size() * sizeof(TPassDev)));
    FS_CUDA(cudaMemcpy(sp->tpass, pd.data(), pd.size() * sizeof(TPassDev),
                       cudaMemcpyHostToDevice));
    FS_CUDA(cudaMalloc(&sp->trec, std::max<size_t>(recs.size(), 1) * sizeof(TRecord)));
    if (!recs.empty())
      FS_CUDA(cudaMemcpy(sp->trec, recs.data(), recs.size() * sizeof(TRecord),
                         cudaMemcpyHostToDevice));
  }
  sp->npass = (int)pd.size();
  sp->tbuilt = true;
}

// Window tables of a space for width W (built once, on the host; see
// window_tables_host).
static void build_window_tables(Space* sp, int W) {
  Space::Win& wt = sp->win[W];
  if (wt.built) return;
  std::vector<uint32_t>& orbits = wt.orb_h;
  std::vector<int>& off = wt.off_h;
  std::vector<uint16_t> offs;
  window_tables_host(sp->norb, sp->nocc, W, orbits, off, offs, wt.okey_h);
  FS_CUDA(cudaMalloc(&wt.orbits, std::max<size_t>(orbits.size(), 1) * 4));
  FS_CUDA(cudaMalloc(&wt.off, off.size() * sizeof(int)));
  FS_CUDA(cudaMalloc(&wt.offs, offs.size() * 2));
  if (!orbits.empty())
    FS_CUDA(cudaMemcpy(wt.orbits, orbits.data(), orbits.size() * 4, cudaMemcpyHostToDevice));
  FS_CUDA(cudaMemcpy(wt.off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
  FS_CUDA(cudaMemcpy(wt.offs, offs.data(), offs.size() * 2, cudaMemcpyHostToDevice));
  wt.built = true;
}

// Orbit and record lists regrouped by cluster rank for clusters of 2^b CTAs
// with the blocked layout (built once per space and b).
static void build_window_groups(Space* sp, int W, int b) {
  Space::Win& wt = sp->win[W];
  if (wt.gorb[b]) return;
  std::vector<uint32_t> gorb;
  std::vector<int> goff;
  window_groups_host(wt.orb_h, wt.off_h, wt.okey_h, b, gorb, goff);
  FS_CUDA(cudaMalloc(&wt.gorb[b], std::max<size_t>(gorb.size(), 1) * 4));
  FS_CUDA(cudaMalloc(&wt.goff[b], std::max<size_t>(goff.size(), 1) * sizeof(int)));
  if (!gorb.empty())
    FS_CUDA(cudaMemcpy(wt.gorb[b], gorb.data(), gorb.size() * 4, cudaMemcpyHostToDevice));
  if (!goff.empty())
    FS_CUDA(cudaMemcpy(wt.goff[b], goff.data(), goff.size() * sizeof(int),
                       cudaMemcpyHostToDevice));
}

static void build_tpass_groups(Space* sp, int b) {
  if (sp->tgrec[b] || sp->tpass_h.empty()) return;
  std::vector<TRecord> grec;
  std::vector<int> goff;
  tpass_groups_host(sp->tpass_h, sp->trec_h, sp->rkey_h, b, grec, goff);
  FS_CUDA(cudaMalloc(&sp->tgrec[b], std::max<size_t>(grec.size(), 1) * sizeof(TRecord)));
  FS_CUDA(cudaMalloc(&sp->tgoff[b], std::max<size_t>(goff.size(), 1) * sizeof(int)));
  if (!grec.empty())
    FS_CUDA(cudaMemcpy(sp->tgrec[b], grec.data(), grec.size() * sizeof(TRecord),
                       cudaMemcpyHostToDevice));
  if (!goff.empty())
    FS_CUDA(cudaMemcpy(sp->tgoff[b], goff.data(), goff.size() * sizeof(int),
                       cudaMemcpyHostToDevice));
}

template <int... U>
static bool seq_equal(useq<U...>, const std::vector<int>& u) {
  constexpr int a[] = {U...};
  if (u.size() != sizeof...(U)) return false;
  for (size_t i = 0; i < u.size(); ++i)
    if (a[i] != u[i]) return false;
  return true;
}
template <int W, size_t... I>
static int match_pattern_w(const std::vector<int>& u, std::index_sequence<I...>) {
  int r = -1;
  ((r < 0 && seq_equal(typename std::tuple_element<I, typename WinPatterns<W>::list>::type{}, u)
        ? (r = (int)I)
        : 0),
   ...);
  return r;
}
// Index of the window pattern equal to the u-sequence u, or -1.
static int match_pattern(int W, const std::vector<int>& u) {
  switch (W) {
    case 4: return match_pattern_w<4>(u, std::make_index_sequence<(size_t)win_npat<4>()>{});
    case 5: return match_pattern_w<5>(u, std::make_index_sequence<(size_t)win_npat<5>()>{});
    case 6: return match_pattern_w<6>(u, std::make_index_sequence<(size_t)win_npat<6>()>{});
    default: return -1;
  }
}

template <typename R>
static WProg<R> make_wprog(const RotProgram& rp, int N, int W) {
  WProg<R> w;
  std::vector<WinStep> steps = schedule_windows(rp, N, W);
  int ng = 0;
  for (size_t st = 0; st < steps.size(); ++st) {
    w.a[st] = (int8_t)steps[st].a;
    w.g0[st] = (int16_t)ng;
    std::vector<int> useq_host;
    for (int k : steps[st].givens) useq_host.push_back(rp.g[k].p - steps[st].a);
    w.pat[st] = (int8_t)match_pattern(W, useq_host);
    for (int k : steps[st].givens) {
      w.u[ng] = (int8_t)(rp.g[k].p - steps[st].a);
      w.set(ng, rp.g[k].c, rp.g[k].s.real(), rp.g[k].s.imag());
      ++ng;
    }
  }
  w.nsteps = (int)steps.size();
  w.g0[w.nsteps] = (int16_t)ng;
  return w;
}

template <typename R>
static GProg<R> make_prog(const RotProgram& rp) {
  GProg<R> p;
  p.m = (int)rp.g.size();
  for (int k = 0; k < p.m; ++k) {
    p.p[k] = (int8_t)rp.g[k].p;
    p.c[k] = (R)rp.g[k].c;
    p.sr[k] = (R)rp.g[k].s.real();
    p.si[k] = (R)rp.g[k].s.imag();
  }
  return p;
}

static void set_window_geom(SweepGeom& g, Space* sp, int W) {
  build_window_tables(sp, W);
  const Space::Win& wt = sp->win[W];
  g.orbits = wt.orbits;
  g.orb_off = wt.off;
  if (g.blocked) {
    build_window_groups(sp, W, g.lgcs);
    g.orb_grp = wt.gorb[g.lgcs];
    g.orb_goff = wt.goff[g.lgcs];
  }
  g.offs = wt.offs;
  g.offs_stride = (sp->nocc + 1) << W;
}

// Kernel choice: window sweeps when the orbitals allow a window; forward
// sweeps on 256 threads when a slab is small enough for two CTAs per SM
// (their window-step barriers then overlap), else 512; reverse sweeps with
// both states of an orbit in one thread (complex64 in one CTA: W = 6;
// clusters: W = 5), complex128 in one CTA in split mode (one half-CTA per
// state, W = 5).
// Gather indices of the tensor-core steps (see TcSeg), built once per space:
// b = 0 for the whole orbit list of each window position, b = 1 for the two
// rank groups of 2-CTA blocked clusters.  Row o of class m holds the
// addresses R_O + F[a][c_lo][S] of the orbit's strings, S in ascending
// local-mask order (the order of the compound matrices).
static void build_tc_index(Space* sp, int b) {
  Space::Win& wt = sp->win[tc::kW];
  if (wt.tc_seg[b]) return;
  const int W = tc::kW, N = sp->norb, n = sp->nocc;
  const int npos = N - W + 1;
  const int ranks = 1 << b;
  // in-window rank offsets F, as in window_tables_host
  std::vector<uint32_t> orbits;
  std::vector<int> off;
  std::vector<uint16_t> offs;
  std::vector<uint8_t> okey;
  window_tables_host(N, n, W, orbits, off, offs, okey);
  std::vector<uint32_t> gorb;
  std::vector<int> goff;
  if (b > 0) window_groups_host(orbits, off, okey, b, gorb, goff);
  static const int order[5] = {3, 2, 4, 1, 5};
  std::vector<uint16_t> idx;
  std::vector<TcSeg> seg((size_t)npos * ranks);
  int mx = 0;
  for (int a = 0; a < npos; ++a)
    for (int r = 0; r < ranks; ++r) {
      const uint32_t* list = b ? gorb.data() : orbits.data();
      const int lo = b ? goff[a * 9 + r] : off[a], hi = b ? goff[a * 9 + r + 1] : off[a + 1];
      TcSeg& sg = seg[(size_t)a * ranks + r];
      sg.start = (int)idx.size();
      for (int i = 0; i < 5; ++i) {
        const int m = order[i];
        const int ns = (int)cbinom(W, m), pad = (ns + 7) / 8 * 8;
        int cnt = 0;
        for (int k = lo; k < hi; ++k) {
          const uint32_t desc = list[k];
          if ((int)(desc >> 24) != m) continue;
          const int RO = desc & 0xFFFF, clo = (desc >> 16) & 0xFF;
          const uint16_t* Fc = offs.data() + (((size_t)a * (n + 1) + clo) << W);
          for (int j = 0; j < pad; ++j)
            idx.push_back(j < ns ? (uint16_t)(RO + Fc[win_mask(W, m, j)]) : (uint16_t)0);
          ++cnt;
        }
        sg.cnt[i] = cnt;
      }
      while (idx.size() % 8) idx.push_back(0);
      sg.len = (int)idx.size() - sg.start;
      sg.pad_ = 0;
      mx = std::max(mx, 2 * sg.len);
    }
  FS_CUDA(cudaMalloc(&wt.tc_idx[b], std::max<size_t>(idx.size(), 8) * sizeof(uint16_t)));
  if (!idx.empty())
    FS_CUDA(cudaMemcpy(wt.tc_idx[b], idx.data(), idx.size() * sizeof(uint16_t),
                       cudaMemcpyHostToDevice));
  FS_CUDA(cudaMalloc(&wt.tc_seg[b], seg.size() * sizeof(TcSeg)));
  FS_CUDA(cudaMemcpy(wt.tc_seg[b], seg.data(), seg.size() * sizeof(TcSeg),
                     cudaMemcpyHostToDevice));
  wt.tc_seg_max[b] = (mx + 15) / 16 * 16;
}

// Tensor-core sweep of one program (complex64, W = 6, 1 or 2 CTAs per
// vector): the step images are built on the device first, into context
// scratch that the sweep then reads (stream order keeps consecutive sweeps
// apart).
template <int NST, bool VJP>
static void dispatch_tc(Ctx* ctx, Space* sthis, int CS, const SweepGeom& g0, const RotProgram& rp,
                        const Mat& X, int nslabs, size_t smem, cudaStream_t st) {
  SweepGeom g = g0;
  set_window_geom(g, sthis, tc::kW);
  Space::Win& wt = sthis->win[tc::kW];
  build_tc_index(sthis, 0);
  g.tc_seg_full = wt.tc_seg[0];
  g.tc_idx_full = wt.tc_idx[0];
  if (CS > 1) {
    build_tc_index(sthis, 1);
    g.tc_seg_grp = wt.tc_seg[1];
    g.tc_idx_grp = wt.tc_idx[1];
  }
  const WProg<double> wpd = make_wprog<double>(rp, sthis->norb, tc::kW);
  const WProg<float> wpf = make_wprog<float>(rp, sthis->norb, tc::kW);
  unsigned char* img = (unsigned char*)scratch(
      ctx, "tc_steps", (size_t)std::max(1, wpd.nsteps) * tc::kStepBytes);
  if (wpd.nsteps > 0) {
    ProfScope ps("tc_step_images", st);
    k_tc_bmats<<<wpd.nsteps, 256, 0, st>>>(wpd, img);
    FS_CUDA(cudaGetLastError());
  }
  g.tc_b = img;
  if (CS == 1)
    launch_sweep_t<float, 1, NST, VJP, tc::kW, tc::kThreads, false, WProg<float>, true>(
        g, wpf, X, nslabs, smem, st);
  else
    launch_sweep_t<float, 2, NST, VJP, tc::kW, tc::kThreads, false, WProg<float>, true>(
        g, wpf, X, nslabs, smem, st);
}

template <typename R, int NST, bool VJP>
static void dispatch_prog(Space* sthis, int CS, const SweepGeom& g0, const RotProgram& rp,
                          const Mat& X, int nslabs, size_t smem, bool two_per_sm,
                          cudaStream_t st) {
  if constexpr (NST == 1) {
    constexpr int W = window_width<R, 1>();
    if (sthis->norb >= W && sthis->dim > 1) {
      SweepGeom g = g0;
      set_window_geom(g, sthis, W);
      auto prog = make_wprog<R>(rp, sthis->norb, W);
      if constexpr (sizeof(R) == 4) {
        // slabs of an even number of vectors: packed vector pairs
        if (CS == 1 && g.lgKV >= 1) {
          if (two_per_sm)
            launch_sweep_t<R, 1, 1, false, W, 256, false, WProg<R>, false, true>(g, prog, X,
                                                                               nslabs, smem, st);
          else
            launch_sweep_t<R, 1, 1, false, W, 512, false, WProg<R>, false, true>(g, prog, X,
                                                                               nslabs, smem, st);
          return;
        }
      }
      if (two_per_sm)
        dispatch_cs<R, NST, VJP, W, 256>(CS, g, prog, X, nslabs, smem, st);
      else
        dispatch_cs<R, NST, VJP, W, 512>(CS, g, prog, X, nslabs, smem, st);
      return;
    }
  } else {
    constexpr int WS = window_width<R, 1>();
    constexpr int WJ = window_width<R, 2>();
    if (CS == 1 && sthis->norb >= WS && sthis->dim > 1) {
      SweepGeom g = g0;
      set_window_geom(g, sthis, WS);
      auto prog = make_wprog<R>(rp, sthis->norb, WS);
      if constexpr (sizeof(R) == 4)
        // complex64: psi and g of an orbit in one thread, packed per string
        // (W = 6; shared addresses and coefficients, two-lane updates)
        launch_sweep_t<R, 1, NST, VJP, WS, 512, false, WProg<R>, false, true>(g, prog, X, nslabs,
                                                                              smem, st);
      else
        launch_sweep_t<R, 1, NST, VJP, WS, 512, true>(g, prog, X, nslabs, smem, st);
      return;
    }
    if (sthis->norb >= WJ && sthis->dim > 1) {
      SweepGeom g = g0;
      set_window_geom(g, sthis, WJ);
      auto prog = make_wprog<R>(rp, sthis->norb, WJ);
      dispatch_cs<R, NST, VJP, WJ, 512>(CS, g, prog, X, nslabs, smem, st);
      return;
    }
  }
  auto prog = make_prog<R>(rp);
  dispatch_cs<R, NST, VJP, 0, 512>(CS, g0, prog, X, nslabs, smem, st);
}

// Split of each vector over the CS ranks of a cluster.  Preferred: rank r
// holds the strings whose occupation of the top b = log2(CS) orbitals reads
// r (a contiguous address range of C(N - b, n - popcount(r)) strings), so
// that the orbits of windows and subsets clear of those orbitals stay
// within one CTA; else (the largest such block does not fit) equal chunks.
template <typename Fits>
static void set_cluster_layout(SweepGeom& g, const Space* sp, int CS, Fits&& fits) {
  g.blocked = 0;
  g.lgcs = 0;
  g.cb[0] = 0;
  if (CS > 1) {
    int b = 0;
    while ((1 << b) < CS) ++b;
    int64_t mx = 0;
    std::vector<int64_t> bs(CS);
    for (int r = 0; r < CS; ++r) {
      const int k = sp->nocc - __builtin_popcount(r);
      bs[r] = (k < 0 || k > sp->norb - b) ? 0 : (int64_t)binom_host(sp->norb - b, k);
      mx = std::max(mx, bs[r]);
    }
    if (sp->norb >= 3 && b <= 3 && fits((int)mx)) {
      g.blocked = 1;
      g.lgcs = b;
      g.chunk = (int)mx;
      for (int r = 0; r < CS; ++r) g.cb[r + 1] = g.cb[r] + (int)bs[r];
      return;
    }
  }
  g.chunk = (g.d + CS - 1) / CS;
  for (int r = 1; r <= CS; ++r) g.cb[r] = std::min(g.d, r * g.chunk);
}

void launch_sweep(Ctx* ctx, const Space* sa, const Space* sb, int dir, void* st0,
                  void* st1, int nst, int dtype, const RotProgram& rp,
                  const PhaseDev& ph, cudaStream_t st, const RevArgs* rev) {
  FS_REQUIRE((nst == 2) == (rev != nullptr), FS_ERR_ARG, "reverse mode needs two states");
  const Space* sthis = dir == 0 ? sa : sb;
  const Space* sother = dir == 0 ? sb : sa;
  FS_REQUIRE(sthis->dim <= kMaxSweepDim, FS_ERR_UNSUPPORTED,
             "string dimension above 65535 is not supported by the sweep kernels");
  FS_REQUIRE((int)rp.g.size() <= kMaxGivens, FS_ERR_ARG, "too many Givens rotations");
  SweepGeom g{};
  g.st[0] = st0;
  g.st[1] = st1;
  g.d_b = sb->dim;
  g.dir = dir;
  g.d = (int)sthis->dim;
  g.nvec = (int)sother->dim;
  g.pairs = sthis->pairs;
  g.npp = sthis->npp;
  g.masks_this = sthis->masks;
  g.masks_other = sother->masks;
  g.norb = sthis->norb;
  g.nchunk = (sthis->norb + 7) / 8;
  g.ea_this = dir == 0 ? ph.ea_a : ph.ea_b;
  g.ea_other = dir == 0 ? ph.ea_b : ph.ea_a;
  g.has_x = ph.has_x;
  if (rev) {
    g.ea2_this = dir == 0 ? rev->ea2_a : rev->ea2_b;
    g.ea2_other = dir == 0 ? rev->ea2_b : rev->ea2_a;
    g.xpairs = sthis->xpairs;
    g.xsign = sthis->xsign;
    g.xcount = sthis->xcount;
    g.nx = sthis->nx;
    g.T = sthis->nx > 0 ? rev->T : nullptr;
    g.W = rev->W;
    if (g.T && sthis->norb >= 4 && sthis->nocc >= 1) {
      build_tpass_tables(const_cast<Space*>(sthis));
      g.tpass = sthis->tpass;
      g.trec = sthis->trec;
      g.npass = sthis->npass;
    }
  }
  g.status = ctx->d_status;
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  const size_t maxsm = (size_t)ctx->prop.sharedMemPerBlockOptin;
  const size_t tab_per_kv = ph.has_x ? g.nchunk * 256 * csz : 0;
  const size_t fixed = ph.has_x ? kMaxOrb * sizeof(double) : 0;
  const size_t tsum = (size_t)g.npass * 32 * (csz / 2);  // per-CTA pass sums
  auto smem_for = [&](int CS, int KV) {
    size_t chunk = (g.d + CS - 1) / CS;
    return (size_t)KV * (chunk * csz * nst + tab_per_kv + fixed) + tsum;
  };
  // tensor-core window steps: complex64, a window of 6 orbitals, the vector
  // on 1 CTA or a blocked pair (the step images take 2 x 35 KB)
  if (dtype == FS_C64 && ctx->sweep_engine == FS_SWEEP_TENSOR && sthis->norb >= tc::kW &&
      sthis->dim > 1 && ctx->prop.major >= 10) {
    Space* sw0 = const_cast<Space*>(sthis);
    build_tc_index(sw0, 0);
    for (int CS = 1; CS <= 2; CS *= 2) {
      if (CS > 1) build_tc_index(sw0, 1);
      const Space::Win& wt = sthis->win[tc::kW];
      const int cap = CS > 1 ? std::max(wt.tc_seg_max[0], wt.tc_seg_max[1]) : wt.tc_seg_max[0];
      auto smem_tc = [&](size_t chunk, int KV) {
        return (size_t)KV * chunk * csz * nst +
               std::max<size_t>(128 + 2 * (size_t)tc::kStepBytes + 2 * (size_t)cap,
                                (size_t)KV * (tab_per_kv + fixed) + tsum);
      };
      SweepGeom gt = g;
      gt.tc_idx_cap = cap;
      set_cluster_layout(gt, sthis, CS, [&](int chunk) { return smem_tc(chunk, 1) <= maxsm; });
      if (CS > 1 && !gt.blocked) continue;
      if (smem_tc(gt.chunk, 1) > maxsm) continue;
      int want = std::max(1, gt.nvec / (2 * ctx->prop.multiProcessorCount));
      int lg = 0;
      while ((2 << lg) <= std::min(want, kMaxKV) && smem_tc(gt.chunk, 2 << lg) <= maxsm) ++lg;
      gt.lgKV = lg;
      if (gt.blocked && gt.npass > 0) {
        build_tpass_groups(const_cast<Space*>(sthis), gt.lgcs);
        gt.trec_grp = sthis->tgrec[gt.lgcs];
        gt.tgoff = sthis->tgoff[gt.lgcs];
      }
      const int KV = 1 << lg;
      const int nslabs = (gt.nvec + KV - 1) / KV;
      // more than half an SM's shared memory: one CTA per SM, so that no two
      // CTAs (of different clusters) ever wait on one SM's tensor memory
      const size_t smem = std::max(smem_tc(gt.chunk, KV),
                                   (size_t)ctx->prop.sharedMemPerMultiprocessor / 2 + 1024);
      Space* sw = const_cast<Space*>(sthis);
      if (nst == 1)
        dispatch_tc<1, false>(ctx, sw, CS, gt, rp, ph.X, nslabs, smem, st);
      else
        dispatch_tc<2, true>(ctx, sw, CS, gt, rp, ph.X, nslabs, smem, st);
      return;
    }
  }
  int CS = 1;
  while (CS <= 8 && smem_for(CS, 1) > maxsm) CS *= 2;
  FS_REQUIRE(CS <= 8, FS_ERR_UNSUPPORTED, "state vector too large for a cluster of 8");
  // two CTAs per SM for single-state sweeps whose slab fits half the SM
  const size_t half_sm = (size_t)ctx->prop.sharedMemPerMultiprocessor / 2 - 1024;
  bool two_per_sm = nst == 1 && CS == 1 && smem_for(1, 1) <= half_sm;
  // complex64 forward sweeps work on packed vector pairs: when only one
  // vector would fit half an SM but two fit the whole, one CTA of 512
  // threads per SM holding two vectors beats two CTAs holding one each
  const bool pair_slab = dtype == FS_C64 && nst == 1 && CS == 1 && g.nvec >= 2 &&
                         smem_for(1, 2) > half_sm && smem_for(1, 2) <= maxsm;
  if (pair_slab) two_per_sm = false;
  const size_t budget = two_per_sm ? half_sm : maxsm;
  // vectors per slab: fit the budget, keep >= 2 slabs per SM when possible
  int want = std::max(1, g.nvec / (2 * ctx->prop.multiProcessorCount));
  int lg = 0;
  while ((2 << lg) <= std::min(want, kMaxKV) && smem_for(CS, 2 << lg) <= budget) ++lg;
  if (pair_slab && lg == 0) lg = 1;
  g.lgKV = lg;
  set_cluster_layout(g, sthis, CS, [&](int chunk) {
    return (size_t)(chunk * csz * nst + tab_per_kv + fixed) + tsum <= maxsm;
  });
  if (g.blocked && g.npass > 0) {
    build_tpass_groups(const_cast<Space*>(sthis), g.lgcs);
    g.trec_grp = sthis->tgrec[g.lgcs];
    g.tgoff = sthis->tgoff[g.lgcs];
  }
  const int KV = 1 << lg;
  const int nslabs = (g.nvec + KV - 1) / KV;
  const size_t smem = std::max<size_t>(
      (size_t)KV * ((size_t)g.chunk * csz * nst + tab_per_kv + fixed) + tsum, 16);
  Space* sw = const_cast<Space*>(sthis);
  if (dtype == FS_C64) {
    if (nst == 1) dispatch_prog<float, 1, false>(sw, CS, g, rp, ph.X, nslabs, smem, two_per_sm, st);
    else dispatch_prog<float, 2, true>(sw, CS, g, rp, ph.X, nslabs, smem, false, st);
  } else {
    if (nst == 1) dispatch_prog<double, 1, false>(sw, CS, g, rp, ph.X, nslabs, smem, two_per_sm, st);
    else dispatch_prog<double, 2, true>(sw, CS, g, rp, ph.X, nslabs, smem, false, st);
  }
}

// ------------------------------------------------------- batched sweeps
size_t wprog_bytes(int dtype) {
  return dtype == FS_C64 ? sizeof(WProg<float>) : sizeof(WProg<double>);
}

int batch_window(int dtype, int nst) {
  return dtype == FS_C64 ? (nst == 1 ? window_width<float, 1>() : window_width<float, 1>())
                         : (nst == 1 ? window_width<double, 1>() : window_width<double, 1>());
}

// One circuit's sweep as a job of a batched launch: one CTA per slab (no
// cluster), window program for the batch window width, slab sized to
// `budget` bytes of shared memory.
// Autotuner of the batched sweeps' slab width: one circuit's sweep as a
// one-job launch of the batched kernel, on scratch states (and scratch W
// and T for the reverse sweeps), for every slab width 2^0 .. 2^lgmax that
// fits the stage's budget; CUDA events on a private stream, the fastest
// mean of two launches after one warm-up wins and is cached per sector and
// sweep kind.  Runs before any capture.
template <typename SmemFor>
static int tune_batch_slab(Ctx* ctx, const SweepGeom& g0, const std::vector<unsigned char>& prog,
                           int nst, int dtype, bool rev, int lgmin, int lgmax,
                           SmemFor&& smem_for, const std::array<int, 8>& key) {
  if (!ctx->tune_stream)
    FS_CUDA(cudaStreamCreateWithFlags(&ctx->tune_stream, cudaStreamNonBlocking));
  cudaStream_t ts = ctx->tune_stream;
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  const size_t nstate = (size_t)g0.d * g0.nvec;
  char* st = (char*)scratch(ctx, "tune_states", nstate * csz * nst);
  FS_CUDA(cudaMemsetAsync(st, 0, nstate * csz * nst, ts));
  // device copies of the program, a zero cross matrix and the job
  char* dev = (char*)scratch(ctx, "tune_job", prog.size() + sizeof(Mat) + sizeof(SweepJob) + 1024);
  char* dprog = dev;
  Mat* dX = (Mat*)(dev + (prog.size() + 255) / 256 * 256);
  SweepJob* djob = (SweepJob*)((char*)dX + (sizeof(Mat) + 255) / 256 * 256);
  int* dcounter = (int*)scratch(ctx, "tune_counter", sizeof(int));
  FS_CUDA(cudaMemcpyAsync(dprog, prog.data(), prog.size(), cudaMemcpyHostToDevice, ts));
  FS_CUDA(cudaMemsetAsync(dX, 0, sizeof(Mat), ts));
  SweepGeom g = g0;
  g.st[0] = st;
  g.st[1] = nst == 2 ? st + nstate * csz : nullptr;
  if (rev) {
    g.T = (double*)scratch(ctx, "tune_T", (size_t)2 * kMaxOrb * kMaxOrb * sizeof(double));
    g.W = g0.W ? scratch(ctx, "tune_W", nstate * (csz / 2)) : nullptr;
  }
  cudaEvent_t e0, e1;
  FS_CUDA(cudaEventCreate(&e0));
  FS_CUDA(cudaEventCreate(&e1));
  std::vector<float> ms(lgmax + 1, 0.f);
  int best = lgmin;
  for (int lg = lgmin; lg <= lgmax; ++lg) {
    g.lgKV = lg;
    SweepJob j{};
    j.g = g;
    j.prog = dprog;
    j.X = dX;
    j.item0 = 0;
    const int nslabs = (g.nvec + (1 << lg) - 1) >> lg;
    const size_t smem = smem_for(1 << lg);
    FS_CUDA(cudaMemcpyAsync(djob, &j, sizeof(j), cudaMemcpyHostToDevice, ts));
    const bool pk = lgmin > 0;
    launch_sweep_batch(ctx, dtype, nst, nullptr, 0, 0, nullptr, smem, ts, pk);  // attribute
    float tot = 0;
    for (int r = 0; r < 3; ++r) {
      FS_CUDA(cudaMemsetAsync(dcounter, 0, sizeof(int), ts));
      if (r == 1) FS_CUDA(cudaEventRecord(e0, ts));
      launch_sweep_batch(ctx, dtype, nst, djob, 1, nslabs, dcounter, smem, ts, pk);
    }
    FS_CUDA(cudaEventRecord(e1, ts));
    FS_CUDA(cudaEventSynchronize(e1));
    FS_CUDA(cudaEventElapsedTime(&tot, e0, e1));
    ms[lg] = tot / 2;
    if (ms[lg] < ms[best]) best = lg;
  }
  FS_CUDA(cudaEventDestroy(e0));
  FS_CUDA(cudaEventDestroy(e1));
  ctx->sweep_tune[key] = best;
  ctx->sweep_tune_ms[key] = ms;
  return best;
}

void plan_batch_sweep(Ctx* ctx, Space* sa, Space* sb, int dir, void* st0, void* st1, int nst,
                      int dtype, const RotProgram& rp, const PhaseDev& ph, const RevArgs* rev,
                      size_t budget, BatchSweepPlan& out) {
  Space* sthis = dir == 0 ? sa : sb;
  Space* sother = dir == 0 ? sb : sa;
  const int W = batch_window(dtype, nst);
  FS_REQUIRE(sthis->norb >= W && sthis->dim > 1 && sthis->dim <= kMaxSweepDim,
             FS_ERR_UNSUPPORTED, "batched sweeps need norb >= 6 and 2 <= dim <= 65535");
  SweepGeom& g = out.g;
  g = SweepGeom{};
  g.st[0] = st0;
  g.st[1] = st1;
  g.d_b = sb->dim;
  g.dir = dir;
  g.d = (int)sthis->dim;
  g.nvec = (int)sother->dim;
  g.pairs = sthis->pairs;
  g.npp = sthis->npp;
  g.masks_this = sthis->masks;
  g.masks_other = sother->masks;
  g.norb = sthis->norb;
  g.nchunk = (sthis->norb + 7) / 8;
  g.ea_this = dir == 0 ? ph.ea_a : ph.ea_b;
  g.ea_other = dir == 0 ? ph.ea_b : ph.ea_a;
  g.has_x = ph.has_x;
  if (rev) {
    g.ea2_this = dir == 0 ? rev->ea2_a : rev->ea2_b;
    g.ea2_other = dir == 0 ? rev->ea2_b : rev->ea2_a;
    g.T = rev->T;
    g.W = rev->W;
    build_tpass_tables(sthis);
    g.tpass = sthis->tpass;
    g.trec = sthis->trec;
    g.npass = sthis->npass;
  }
  set_window_geom(g, sthis, W);
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  const size_t tab_per_kv = ph.has_x ? g.nchunk * 256 * csz : 0;
  const size_t fixed = ph.has_x ? kMaxOrb * sizeof(double) : 0;
  const size_t tsum = (size_t)g.npass * 32 * (csz / 2);
  auto smem_for = [&](int KV) {
    return (size_t)KV * ((size_t)g.d * csz * nst + tab_per_kv + fixed) + tsum;
  };
  FS_REQUIRE(smem_for(1) <= budget, FS_ERR_UNSUPPORTED, "batched sweep slab does not fit");
  g.chunk = g.d;
  g.cb[0] = 0;
  g.cb[1] = g.d;
  out.prog.resize(wprog_bytes(dtype));
  if (dtype == FS_C64) {
    auto w = make_wprog<float>(rp, sthis->norb, W);
    memcpy(out.prog.data(), &w, sizeof(w));
  } else {
    auto w = make_wprog<double>(rp, sthis->norb, W);
    memcpy(out.prog.data(), &w, sizeof(w));
  }
  // slab width: the widest that fits the budget (at most 64 vectors), or the
  // autotuned width for this sector and sweep kind
  int lgmax = 0;
  while ((2 << lgmax) <= std::min(g.nvec, kMaxKV) && smem_for(2 << lgmax) <= budget) ++lgmax;
  // complex64 forward sweeps: at least two vectors per slab, run as packed
  // vector pairs
  const int lgmin = dtype == FS_C64 && nst == 1 && lgmax >= 1 ? 1 : 0;
  const std::array<int, 8> key = {sthis->norb, sthis->nocc, sother->nocc, dtype, nst,
                                  rev != nullptr, ph.has_x, (int)(budget >> 10)};
  int lg = -1;
  auto it = ctx->sweep_tune.find(key);
  if (it != ctx->sweep_tune.end()) {
    lg = std::min(it->second, lgmax);
  } else if (ctx->batch_tuning && lgmax > lgmin) {
    lg = tune_batch_slab(ctx, g, out.prog, nst, dtype, rev != nullptr, lgmin, lgmax, smem_for,
                         key);
  }
  if (lg < 0) {  // untuned: about eight slabs per circuit
    const int want = std::max(1, g.nvec / 8);
    lg = 0;
    while ((2 << lg) <= std::min(want, kMaxKV) && lg < lgmax) ++lg;
  }
  lg = std::max(lg, lgmin);
  g.lgKV = lg;
  out.nslabs = (g.nvec + (1 << lg) - 1) >> lg;
  out.smem = smem_for(1 << lg);
  out.pk = lgmin > 0;
}

void launch_sweep_batch(Ctx* ctx, int dtype, int nst, const SweepJob* jobs, int njobs, int total,
                        int* counter, size_t smem, cudaStream_t st, bool pk) {
  const int sms = ctx->prop.multiProcessorCount;
  const size_t half_sm = (size_t)ctx->prop.sharedMemPerMultiprocessor / 2 - 1024;
  if (dtype == FS_C64) {
    constexpr int W = window_width<float, 1>();
    if (nst == 1 && pk) {
      if (smem <= half_sm)
        launch_batch_t<float, 1, false, W, 256, false, true>(jobs, njobs, total, counter, smem, 2 * sms, st);
      else
        launch_batch_t<float, 1, false, W, 512, false, true>(jobs, njobs, total, counter, smem, sms, st);
    } else if (nst == 1) {
      if (smem <= half_sm)
        launch_batch_t<float, 1, false, W, 256, false>(jobs, njobs, total, counter, smem, 2 * sms, st);
      else
        launch_batch_t<float, 1, false, W, 512, false>(jobs, njobs, total, counter, smem, sms, st);
    } else {
      // psi and g packed per string, one thread per orbit of both
      launch_batch_t<float, 2, true, W, 512, false, true>(jobs, njobs, total, counter, smem, sms, st);
    }
  } else {
    constexpr int W = window_width<double, 1>();
    if (nst == 1) {
      if (smem <= half_sm)
        launch_batch_t<double, 1, false, W, 256, false>(jobs, njobs, total, counter, smem, 2 * sms, st);
      else
        launch_batch_t<double, 1, false, W, 512, false>(jobs, njobs, total, counter, smem, sms, st);
    } else {
      launch_batch_t<double, 2, true, W, 512, true>(jobs, njobs, total, counter, smem, sms, st);
    }
  }
}

// ------------------------------------------------------------------ phase
// One streaming pass: psi[i][j] *= ea_a[i] ea_b[j] exp(i sum X[p][q]) with
// the cross tables built per row from the alpha string.
template <typename R>
__global__ void __launch_bounds__(256)
    k_phase(cx_t<R>* vec, int64_t da, int64_t db, const uint32_t* ma,
            const uint32_t* mb, int norb, int nchunk, const void* ea_a,
            const void* ea_b, int has_x, const __grid_constant__ Mat X) {
  using C = cx_t<R>;
  __shared__ double w[kMaxOrb];
  __shared__ C tab[4 * 256];
  SweepGeom g{};
  g.dir = 1;
  g.norb = norb;
  g.nchunk = nchunk;
  g.has_x = has_x;
  g.masks_other = ma;
  for (int64_t i = blockIdx.x; i < da; i += gridDim.x) {
    C fa = ld_ea<R>(ea_a, i);
    if (has_x) {
      __syncthreads();
      build_cross_tables<R>(g, X, (int)i, 1, w, tab, threadIdx.x, blockDim.x);
    }
    C* row = vec + i * db;
    for (int64_t j = threadIdx.x; j < db; j += blockDim.x) {
      C f = cmul<R>(fa, ld_ea<R>(ea_b, j));
      if (has_x) {
        uint32_t m = __ldg(mb + j);
        for (int c = 0; c < nchunk; ++c) f = cmul<R>(f, tab[c * 256 + ((m >> (8 * c)) & 255)]);
      }
      row[j] = cmul<R>(f, row[j]);
    }
  }
}

void launch_phase(const Space* sa, const Space* sb, void* vec, int dtype,
                  const PhaseDev& ph, cudaStream_t st) {
  ProfScope ps(dtype == FS_C64 ? "phase_f32" : "phase_f64", st);
  int nchunk = (sa->norb + 7) / 8;
  unsigned grid = (unsigned)std::min<int64_t>(sa->dim, 4096);
  if (dtype == FS_C64)
    k_phase<float><<<grid, 256, 0, st>>>((float2*)vec, sa->dim, sb->dim, sa->masks,
                                         sb->masks, sa->norb, nchunk, ph.ea_a,
                                         ph.ea_b, ph.has_x, ph.X);
  else
    k_phase<double><<<grid, 256, 0, st>>>((double2*)vec, sa->dim, sb->dim, sa->masks,
                                          sb->masks, sa->norb, nchunk, ph.ea_a,
                                          ph.ea_b, ph.has_x, ph.X);
  FS_CUDA(cudaGetLastError());
}

// Per-string factors (FP64 arithmetic, stored in the state precision).
template <typename R>
__global__ void k_string_phase(cx_t<R>* out, const uint32_t* masks, int64_t dim,
                               int norb, const __grid_constant__ StrPhase f) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= dim) return;
  uint32_t m = masks[e];
  double re = 1, im = 0, ang = 0;
  for (int p = 0; p < norb; ++p) {
    if (!((m >> p) & 1u)) continue;
    if (f.use_d) {
      double dr = f.d[2 * p], di = f.d[2 * p + 1];
      double nr = re * dr - im * di;
      im = re * di + im * dr;
      re = nr;
    }
    if (f.use_lam) ang -= f.t * f.lam[p];
    if (f.use_j)
      for (int q = 0; q < norb; ++q)
        if ((m >> q) & 1u) ang -= 0.5 * f.t * f.J.v[p * norb + q];
  }
  double r = ang - 6.283185307179586 * rint(ang * 0.15915494309189535);
  double s, c;
  sincos(r, &s, &c);
  out[e] = mk<R>((R)(re * c - im * s), (R)(re * s + im * c));
}

void preload_phase_kernels() {
  cudaFuncAttributes fa;
  FS_CUDA(cudaFuncGetAttributes(&fa, k_string_phase<float>));
  FS_CUDA(cudaFuncGetAttributes(&fa, k_string_phase<double>));
  FS_CUDA(cudaFuncGetAttributes(&fa, k_phase<float>));
  FS_CUDA(cudaFuncGetAttributes(&fa, k_phase<double>));
}

void launch_string_phase(const Space* sp, void* out, int dtype, const StrPhase& f,
                         cudaStream_t st) {
  ProfScope ps("string_phase", st);
  unsigned grid = (unsigned)((sp->dim + 127) / 128);
  if (dtype == FS_C64)
    k_string_phase<float><<<grid, 128, 0, st>>>((float2*)out, sp->masks, sp->dim,
                                                 sp->norb, f);
  else
    k_string_phase<double><<<grid, 128, 0, st>>>((double2*)out, sp->masks, sp->dim,
                                                  sp->norb, f);
  FS_CUDA(cudaGetLastError());
}

// ----------------------------------------------- Hartree-Fock closed form
// v[e] = det(R[I_e, 0..n-1]) by Gaussian elimination with partial pivoting,
// FP64.
__global__ void k_slater_minors(const uint32_t* masks, int64_t dim, int norb, int n,
                                const __grid_constant__ CMat R, double2* v) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= dim) return;
  v[e] = slater_minor(masks[e], norb, n, R.v);
}

template <typename R>
__global__ void k_outer(cx_t<R>* vec, const double2* va, const double2* vb, int64_t da,
                        int64_t db) {
  int64_t n = da * db;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = k / db, j = k - i * db;
    double2 a = va[i], b = vb[j];
    vec[k] = mk<R>((R)(a.x * b.x - a.y * b.y), (R)(a.x * b.y + a.y * b.x));
  }
}

void launch_slater(Ctx* ctx, const Space* sa, const Space* sb, void* vec, int dtype,
                   const CMat& R, cudaStream_t st) {
  ProfScope ps("slater", st, 3);
  double2* va = (double2*)scratch(ctx, "slater_a", sa->dim * 16);
  double2* vb = (double2*)scratch(ctx, "slater_b", sb->dim * 16);
  k_slater_minors<<<(unsigned)((sa->dim + 63) / 64), 64, 0, st>>>(
      sa->masks, sa->dim, sa->norb, sa->nocc, R, va);
  FS_CUDA(cudaGetLastError());
  k_slater_minors<<<(unsigned)((sb->dim + 63) / 64), 64, 0, st>>>(
      sb->masks, sb->dim, sb->norb, sb->nocc, R, vb);
  FS_CUDA(cudaGetLastError());
  int64_t n = sa->dim * sb->dim;
  unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32);
  if (dtype == FS_C64)
    k_outer<float><<<grid, 256, 0, st>>>((float2*)vec, va, vb, sa->dim, sb->dim);
  else
    k_outer<double><<<grid, 256, 0, st>>>((double2*)vec, va, vb, sa->dim, sb->dim);
  FS_CUDA(cudaGetLastError());
}

}  // namespace fs
