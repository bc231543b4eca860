// Host side of libfif.so: plan lifetime, per-length schedules and tables,
// argument validation, and the C entry points declared in include/fif.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <vector>

#include "fif_internal.h"

using namespace fif;

struct LargeTables;
struct LargeBuffers;

namespace {

struct LengthTables {
  FftSched sched;
  float2* tw = nullptr;
  float2* tw_lo = nullptr;
  float2* wtab = nullptr;
  double* sin64 = nullptr;
  double* om64 = nullptr;  // shape window only
  int* ltab = nullptr;     // mask length per extrema count (FftSched::ltab)
  float2* gtab = nullptr;  // multipliers of m = max_inner per (L, k) (fused path; built lazily)
  std::map<std::vector<int>, float2*> ptw;  // per-pass twiddles per fused radix sequence
};

struct BatchLayout {
  std::vector<int64_t> offsets, out_offsets;
  struct LargeCls {
    int64_t n;
    int count;
    LargeTables* lt;
    LargeBuffers* b;
  };
  std::vector<LargeCls> lcls;
  // CUDA graph of the whole call, valid for the pointers in key
  cudaGraphExec_t exec = nullptr;
  const void* key[8] = {nullptr};
  // classes: contiguous ranges of the sorted signal list sharing one length
  struct Cls {
    int first, count, smem, threads, grid, E, n;
    bool tc;  // split-BF16 tensor-core radix-16 passes (E = 16)
  };
  std::vector<Cls> classes;
  SigDesc* d_sigs = nullptr;
  FftSched* d_scheds = nullptr;
  int* d_counters = nullptr;
};

}  // namespace

struct LargeTables {
  LgSched G;
  std::vector<void*> allocs;
  std::map<std::vector<int>, float2*> ptw;  // per-pass twiddles per (R, radix sequence)
};

// The per-pass twiddle tables of the FP32 levels' sub-FFT schedules (global
// memory, read through L1, in place of the folded shared-memory table), built
// once per (R, radix sequence) and owned by lt.
static cudaError_t large_pass_tables(LargeTables& lt, LgSched& G, cudaStream_t st) {
  for (FftSched* s : {&G.S1, &G.S2}) {
    std::vector<int> key{s->n};
    key.insert(key.end(), s->radix, s->radix + s->npass);
    auto it = lt.ptw.find(key);
    if (it == lt.ptw.end()) {
      float2* d = nullptr;
      cudaError_t e = cudaMalloc(&d, sizeof(float2) * (size_t)std::max(s->Nc - 1, 1));
      if (e == cudaSuccess) e = build_pass_twiddles(*s, d, st);
      if (e != cudaSuccess) {
        cudaFree(d);
        return e;
      }
      it = lt.ptw.emplace(key, d).first;
    }
    s->ptw = it->second;
  }
  return cudaSuccess;
}

struct LargeBuffers {
  int64_t n = 0;
  int cap = 0;                 // signals the buffers hold
  std::vector<void*> allocs;
  float4* za = nullptr;
  float4* zb = nullptr;
  float2* spec = nullptr;
  float2* work = nullptr;
  float2* work2 = nullptr;
  float* rem = nullptr;
  float* rem2 = nullptr;
  float2* row = nullptr;
  int* st = nullptr;
  unsigned char* part = nullptr;
  double* om64 = nullptr;  // shape window rows
  LgSig* d_sigs = nullptr;
};

struct fif_plan_s {
  fif_plan_desc desc;
  MethodParams mp;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int smem_optin = 0;
  std::map<int64_t, LengthTables> tables;
  StagedScratch scr{};
  int64_t scr_n = 0;
  BatchLayout layout;
  bool layout_valid = false;
  // host-buffer entry point staging
  void* h2d_buf = nullptr;
  size_t h2d_cap = 0;
  // large-length path
  std::map<int64_t, LargeTables> large;
  std::map<int64_t, LargeBuffers> large_bufs;         // per length, batch layouts
  std::map<int64_t, LargeBuffers> large_single_bufs;  // per length, fif_decompose
  // fused schedules chosen by fif_plan_tune / fif_plan_load_tuning: n -> E
  std::map<int64_t, int> fused_E;
  // multi-pass schedules chosen by fif_plan_tune / fif_plan_load_tuning:
  // n -> {E1, TJ1, E2, TJ2} of the two FP32 inverse levels
  std::map<int64_t, std::array<int, 4>> large_sched;
  // FIF_WIN_SHAPE: the shape's samples (host copy, and on the device)
  std::vector<double> shape;
  double* d_shape = nullptr;
  // branches of the batch graph: one per length class
  static constexpr int kBranches = 8;
  cudaStream_t aux[kBranches] = {nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kBranches] = {nullptr};
};

namespace {

bool is_smooth(int64_t n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

// FFT plan with E elements per thread for a complex FFT of Nc = 2^p 3^q
// points: T = Nc / E threads (at most max_threads), radix passes that all
// divide E (a thread holds E/R butterflies of one pass in registers): the
// factors 3 first (as radix-9 passes when 9 divides E, the odd one left as a
// radix-3 pass; else radix-3 passes), then 2^p as passes of the main radix RM (largest power
// of two dividing E, at most 16) and of RM/2, both kept inline by the kernels
// (p = a log2(RM) + b log2(RM/2) with the fewest passes); a single other
// radix only when no such split exists.  half_first puts the RM/2 passes
// before the RM passes: the first pass (Ns = 1) stores its outputs R points
// apart, so a smaller first radix halves its shared-memory bank conflicts
// (the fused kernel's plans; measured 3 % faster there).
bool plan_with_E(int Nc, int E, int max_threads, FftSched& s, bool half_first = false) {
  int p = 0, q = 0, r = Nc;
  while (r % 2 == 0) r /= 2, p++;
  while (r % 3 == 0) r /= 3, q++;
  if (r != 1 || E < 2 || Nc % E) return false;
  if (q > 0 && E % 3) return false;
  if (p > 0 && E % 2) return false;
  if (E % 2 && E % 3) return false;
  if (Nc / E > max_threads) return false;
  bool known = false;
  for (int k : {2, 3, 4, 6, 8, 9, 12, 16, 18, 24, 27}) known |= k == E;
  if (!known) return false;  // the kernels are instantiated for these E only
  FftSched t = s;
  t.E = E;
  t.T = Nc / E;
  t.npass = 0;
  // the factors 3 first: radix 9 (two radix-3 stages in registers) where E
  // holds nine points, radix 3 otherwise
  if (E % 9 == 0) {
    for (int i = 0; i < q / 2; i++) t.radix[t.npass++] = 9;
    if (q % 2) t.radix[t.npass++] = 3;
  } else {
    for (int i = 0; i < q; i++) t.radix[t.npass++] = 3;
  }
  int lm = 0;
  while (lm < 4 && E % (2 << lm) == 0) lm++;  // RM = 2^lm
  int a = -1, b = 0;
  if (lm >= 2) {
    for (int bb = 0; bb * (lm - 1) <= p; bb++) {
      const int restp = p - bb * (lm - 1);
      if (restp % lm == 0) {
        a = restp / lm;
        b = bb;
        break;
      }
    }
  }
  if (a >= 0) {
    if (t.npass + a + b > kMaxPass) return false;
    if (half_first)
      for (int i = 0; i < b; i++) t.radix[t.npass++] = 1 << (lm - 1);
    for (int i = 0; i < a; i++) t.radix[t.npass++] = 1 << lm;
    if (!half_first)
      for (int i = 0; i < b; i++) t.radix[t.npass++] = 1 << (lm - 1);
  } else {
    int rem2 = 1 << p;
    while (rem2 > 1) {
      int R = 2;
      for (int c : {16, 8, 4}) {
        if (E % c == 0 && rem2 % c == 0) {
          R = c;
          break;
        }
      }
      if (t.npass >= kMaxPass) return false;
      t.radix[t.npass++] = R;
      rem2 /= R;
    }
  }
  s = t;
  return true;
}

// Largest thread count a fused kernel with E elements per thread may run.
int fused_max_threads(int E) { return E <= kWideMaxE ? 1024 : 512; }

// Default FFT plan.  The default order favours large E (at most 512 threads:
// the staged, allocation-free and multi-pass kernels).  The wide order of the
// fused kernel favours E <= 12 with up to 1024 threads (64 registers a
// thread, twice the resident warps; its radix-8 and radix-4 passes fit) and
// falls back to the default order.
bool make_fft_plan(int Nc, FftSched& s, bool wide = false) {
  static const int prefs[] = {16, 24, 12, 18, 9, 27, 8, 6, 4, 3, 2};
  static const int wprefs[] = {8, 12, 6, 9, 16, 24, 18, 27, 4, 3, 2};
  for (int E : wide ? wprefs : prefs)
    if (plan_with_E(Nc, E, wide ? fused_max_threads(E) : 512, s, wide)) return true;
  return false;
}

// The fused kernel's schedule for one length: the tuned E if the plan has
// one, else the wide default, else the length's own plan.
bool fused_plan(const fif_plan_s* p, const FftSched& base, FftSched& out) {
  out = base;
  // the split-BF16 variant runs its radix-16 passes on the tensor cores: E = 16
  // wherever the length has such a schedule (else the FP32 schedule below)
  if (p->desc.precision == FIF_PREC_SPLIT_BF16 &&
      plan_with_E(base.Nc, 16, fused_max_threads(16), out, true))
    return true;
  out = base;
  auto it = p->fused_E.find(base.n);
  if (it != p->fused_E.end() &&
      plan_with_E(base.Nc, it->second, fused_max_threads(it->second), out, true))
    return true;
  out = base;
  FftSched w = base;
  if (make_fft_plan(base.Nc, w, true)) out = w;
  return true;
}

// smem_limit: shared memory per block the fused kernel may use; the folded
// twiddle table goes to shared memory when it fits under that limit.
bool make_sched(int64_t n64, FftSched& s, int smem_limit = 0) {
  if (n64 < 4 || n64 > (1 << 24) || !is_smooth(n64)) return false;
  const int n = (int)n64;
  memset(&s, 0, sizeof(s));
  s.n = n;
  s.odd = n & 1;
  s.Nc = s.odd ? n : n / 2;
  s.P = s.odd ? (n + 1) / 2 : n / 2 + 1;
  s.Lmax = (n + 1) / 2;
  s.tw_fold = n % 8 == 0 ? 3 : n % 4 == 0 ? 2 : n % 2 == 0 ? 1 : 0;
  s.tw_entries = s.tw_fold == 0 ? n : (n >> s.tw_fold) + 1;
  s.tw_shared = 1;
  if (smem_limit > 0 && fused_smem_bytes(s) > (size_t)smem_limit) s.tw_shared = 0;
  return make_fft_plan(s.Nc, s);
}

}  // namespace

// The staged-path schedule of length n (no allocation; host arithmetic only).
bool fif::staged_schedule(int64_t n, FftSched& s) { return make_sched(n, s, 0); }

namespace {

fif_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FIF_OK;
  if (e == cudaErrorMemoryAllocation) return FIF_ENOMEM;
  return FIF_ECUDA;
}

int device_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return v;
}

bool fused_fits(const FftSched& s, int smem_optin) {
  return fused_smem_bytes(s) <= (size_t)smem_optin;
}

bool staged_fits(const FftSched& s, int smem_optin) {
  const size_t work = ((work_points(s) + 1) & ~(size_t)1) * sizeof(float2) +
                      tw_slots(s) * sizeof(float2);
  const size_t ffb = (size_t)s.Nc * 16;
  return (work > ffb ? work : ffb) + 1024 <= (size_t)smem_optin;
}

fif_status get_tables(fif_plan_t p, int64_t n, LengthTables** out) {
  auto it = p->tables.find(n);
  if (it != p->tables.end()) {
    *out = &it->second;
    return FIF_OK;
  }
  LengthTables t;
  if (!make_sched(n, t.sched, p->smem_optin)) return FIF_EUNSUPPORTED;
  const FftSched& s = t.sched;
  cudaError_t e = cudaMalloc(&t.tw, sizeof(float2) * (size_t)s.n);
  if (e == cudaSuccess) e = cudaMalloc(&t.tw_lo, sizeof(float2) * (size_t)s.n);
  if (e == cudaSuccess) e = cudaMalloc(&t.sin64, sizeof(double) * (size_t)(s.n / 2 + 1));
  if (e == cudaSuccess) e = cudaMalloc(&t.wtab, sizeof(float2) * (size_t)s.Lmax * (size_t)s.P);
  if (e == cudaSuccess && p->d_shape)
    e = cudaMalloc(&t.om64, sizeof(double) * (size_t)s.Lmax * (size_t)s.P);
  // (only when every entry fits an int; forced mask lengths read no rule)
  const bool want_ltab = !(p->desc.flags & FIF_FORCE_L) && p->desc.nu * (double)s.n < 1e9;
  if (e == cudaSuccess && want_ltab) e = cudaMalloc(&t.ltab, sizeof(int) * (size_t)(s.n + 1));
  if (e == cudaSuccess && want_ltab) {
    // the outer test's mask rule for every extrema count, in the binary64
    // expression the kernels and the oracle evaluate: mask_scale * floor((nu * n) / k)
    std::vector<int> h((size_t)s.n + 1, 0);
    for (int k = 1; k <= s.n; k++) {
      double v = p->desc.nu * (double)s.n;
      v = v / (double)k;
      h[(size_t)k] = p->desc.mask_scale * (int)floor(v);
    }
    e = cudaMemcpy(t.ltab, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice);
  }
  t.sched.ltab = t.ltab;
  t.sched.tw = t.tw;
  t.sched.tw_lo = t.tw_lo;
  t.sched.wtab = t.wtab;
  t.sched.sin64 = t.sin64;
  t.sched.om64 = t.om64;
  t.sched.om64_stride = s.P;
  if (e == cudaSuccess) {
    if (p->d_shape) {
      e = build_twiddles(s.n, t.tw, t.tw_lo, t.sin64, p->stream);
      if (e == cudaSuccess)
        e = build_shape_window(t.sched, p->d_shape, (int)p->shape.size(), t.wtab, t.om64, p->stream);
    } else {
      e = build_tables(s.n, s.P, s.Lmax, t.tw, t.tw_lo, t.wtab, t.sin64, p->stream);
    }
  }
  if (e != cudaSuccess) {
    cudaFree(t.tw);
    cudaFree(t.tw_lo);
    cudaFree(t.sin64);
    cudaFree(t.wtab);
    cudaFree(t.om64);
    cudaFree(t.ltab);
    cudaGetLastError();
    return cuda_status(e);
  }
  auto res = p->tables.emplace(n, t);
  *out = &res.first->second;
  return FIF_OK;
}

void free_layout(BatchLayout& l) {
  if (l.exec) cudaGraphExecDestroy(l.exec);
  cudaFree(l.d_sigs);
  cudaFree(l.d_scheds);
  cudaFree(l.d_counters);
  l = BatchLayout();
}

// A shape is usable when its samples are finite and >= 0 and its linear
// interpolant is > 0 inside (0, 1), so that every filter tap h_i > 0.
bool shape_valid(const double* g, int32_t len) {
  if (!g || len < 1 || len > 65536) return false;
  for (int32_t j = 0; j < len; j++)
    if (!isfinite(g[j]) || g[j] < 0.0) return false;
  if (len == 1) return g[0] > 0.0;
  if (len == 2) return g[0] + g[1] > 0.0;
  for (int32_t j = 1; j < len - 1; j++)
    if (!(g[j] > 0.0)) return false;
  return true;
}

fif_status validate_desc(const fif_plan_desc* d) {
  if (!d) return FIF_EINVAL;
  if (d->window != FIF_WIN_TRIANGLE && d->window != FIF_WIN_SHAPE) return FIF_EINVAL;
  if (d->window == FIF_WIN_SHAPE) {
    if (!shape_valid(d->window_shape, d->window_shape_len)) return FIF_EINVAL;
    if (d->flags & FIF_APRIORI_N0) return FIF_EUNSUPPORTED;
  }
  if (d->precision != FIF_PREC_FP32 && d->precision != FIF_PREC_SPLIT_BF16) return FIF_EINVAL;
  if (!(d->delta > 0.0) || !isfinite(d->delta)) return FIF_EINVAL;
  if (d->max_inner < 1 || d->max_inner > (1 << 20)) return FIF_EINVAL;
  if (d->max_imfs < 0 || d->max_imfs > kMaxImfs) return FIF_EINVAL;
  if (d->max_n < 4 || d->max_n > (1 << 24)) return FIF_EINVAL;
  if (d->flags & ~(FIF_FORCE_L | FIF_FORCE_MULTIPASS | FIF_APRIORI_N0 | FIF_PEAK_MASK))
    return FIF_EINVAL;
  if (!(d->gamma >= 0.0 && d->gamma < 1.0)) return FIF_EINVAL;
  if (!(d->flags & FIF_FORCE_L)) {
    if (!(d->nu > 0.0) || !isfinite(d->nu)) return FIF_EINVAL;
    if (d->mask_scale < 1 || d->mask_scale > 2) return FIF_EINVAL;
  }
  return FIF_OK;
}

// Sort signals by length (longest first), one class per distinct length, and
// upload the descriptors.  Reused while the same layout is passed again.
// merge: classes with the same E and precision share one persistent launch (a
// single work counter over all their signals, longest first; each signal
// brings its own schedule), sized for the largest member; a length joins a
// launch only while its shared memory is at least half the launch's, so a
// short signal's CTA does not hold the shared memory (and SM slots) of a much
// longer one.  The tuner times every length on its own (merge = false).
fif_status prepare_layout(fif_plan_t p, const int64_t* offsets, const int64_t* out_offsets,
                          int64_t batch, const std::vector<int>& subset, bool merge = true) {
  BatchLayout& l = p->layout;
  free_layout(l);
  p->layout_valid = false;
  // per distinct length: its fused schedule (with its per-pass twiddle table)
  struct LenInfo {
    FftSched fs;
    int smem, threads, sched, group;
    bool tc;
  };
  std::map<int64_t, LenInfo> info;
  std::vector<FftSched> scheds;
  for (int i : subset) {
    const int64_t n = offsets[i + 1] - offsets[i];
    if (info.count(n)) continue;
    LengthTables* t = nullptr;
    fif_status st = get_tables(p, n, &t);
    if (st != FIF_OK) return st;
    // the fused kernel's own FFT plan over the length's tables, with its per-pass
    // twiddle table (global memory, read through L1) in place of the folded
    // shared-memory table
    FftSched fs = t->sched;
    fused_plan(p, t->sched, fs);
    {
      std::vector<int> key(fs.radix, fs.radix + fs.npass);
      auto it = t->ptw.find(key);
      if (it == t->ptw.end()) {
        float2* d = nullptr;
        cudaError_t e = cudaMalloc(&d, sizeof(float2) * (size_t)std::max(fs.Nc - 1, 1));
        if (e == cudaSuccess) e = build_pass_twiddles(fs, d, p->stream);
        if (e != cudaSuccess) {
          cudaFree(d);
          cudaGetLastError();
          return cuda_status(e);
        }
        it = t->ptw.emplace(key, d).first;
      }
      fs.ptw = it->second;
      fs.tw_shared = 0;
    }
    if (!t->gtab) {
      // the multipliers of m = max_inner per (L, k), read by the inverse split
      // step directly whenever the search ends at max_inner
      cudaError_t e = cudaMalloc(&t->gtab, sizeof(float2) * (size_t)fs.Lmax * (size_t)fs.P);
      if (e == cudaSuccess)
        e = build_mult_table(fs.n, fs.P, fs.Lmax, p->desc.max_inner, p->desc.gamma, t->om64,
                             t->gtab, p->stream);
      if (e != cudaSuccess) {
        cudaFree(t->gtab);
        t->gtab = nullptr;
        cudaGetLastError();
        return cuda_status(e);
      }
    }
    fs.gtab = t->gtab;
    LenInfo li;
    li.fs = fs;
    li.smem = (int)fused_smem_bytes(fs);
    li.threads = sched_threads(fs);
    li.sched = (int)scheds.size();
    li.tc = false;
    if (p->desc.precision == FIF_PREC_SPLIT_BF16 && fs.E == 16)
      for (int q = 0; q < fs.npass; q++) li.tc |= fs.radix[q] == 16;
    li.group = 0;
    scheds.push_back(fs);
    info[n] = li;
  }
  // launch groups: lengths longest first; without merging one group per length,
  // else a length joins the first group of its E and precision whose largest
  // shared memory is at most twice its own
  struct Group {
    int E, smem, threads;
    bool tc;
  };
  std::vector<Group> groups;
  for (auto it = info.rbegin(); it != info.rend(); ++it) {
    LenInfo& li = it->second;
    int gsel = -1;
    if (merge)
      for (size_t g = 0; g < groups.size(); g++)
        if (groups[g].E == li.fs.E && groups[g].tc == li.tc && 2 * li.smem >= groups[g].smem) {
          gsel = (int)g;
          break;
        }
    if (gsel < 0) {
      gsel = (int)groups.size();
      groups.push_back(Group{li.fs.E, li.smem, li.threads, li.tc});
    }
    groups[gsel].smem = std::max(groups[gsel].smem, li.smem);
    groups[gsel].threads = std::max(groups[gsel].threads, li.threads);
    li.group = gsel;
  }
  // signals in group order, longest first inside a group
  std::vector<int> order(subset);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int64_t na = offsets[a + 1] - offsets[a], nb = offsets[b + 1] - offsets[b];
    const int ga = info[na].group, gb = info[nb].group;
    return ga != gb ? ga < gb : na > nb;
  });
  const int64_t nfused = (int64_t)order.size();
  std::vector<SigDesc> sigs((size_t)nfused);
  for (int64_t r = 0; r < nfused; r++) {
    const int i = order[(size_t)r];
    const int64_t n = offsets[i + 1] - offsets[i];
    const LenInfo& li = info[n];
    sigs[(size_t)r] = SigDesc{offsets[i], out_offsets[i], li.sched, (int)n, i, 0};
    if (r == 0 || info[(int64_t)sigs[(size_t)r - 1].n].group != li.group) {
      const Group& g = groups[(size_t)li.group];
      l.classes.push_back(BatchLayout::Cls{(int)r, 0, g.smem, g.threads, 0, g.E, (int)n, g.tc});
    }
    l.classes.back().count++;
  }
  for (auto& c : l.classes) {
    const int occ = fused_blocks_per_sm(c.E, c.smem, c.threads, c.tc);
    if (occ <= 0) return FIF_EUNSUPPORTED;
    c.grid = std::min(c.count, occ * p->num_sms);
  }
  cudaError_t e = cudaMalloc(&l.d_sigs, sizeof(SigDesc) * (size_t)std::max<int64_t>(nfused, 1));
  if (e == cudaSuccess) e = cudaMalloc(&l.d_scheds, sizeof(FftSched) * std::max<size_t>(scheds.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc(&l.d_counters, sizeof(int) * std::max<size_t>(l.classes.size(), 1));
  if (e == cudaSuccess && nfused)
    e = cudaMemcpyAsync(l.d_sigs, sigs.data(), sizeof(SigDesc) * (size_t)nfused,
                        cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess && !scheds.empty())
    e = cudaMemcpyAsync(l.d_scheds, scheds.data(), sizeof(FftSched) * scheds.size(),
                        cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    free_layout(l);
    return cuda_status(e);
  }
  l.offsets.assign(offsets, offsets + batch + 1);
  l.out_offsets.assign(out_offsets, out_offsets + batch);
  p->layout_valid = true;
  return FIF_OK;
}

}  // namespace

namespace {

bool make_sub_sched(int R, FftSched& s) {
  memset(&s, 0, sizeof(s));
  s.n = R;
  s.Nc = R;
  s.odd = 1;  // complex transform of R points
  s.P = R;
  s.tw_fold = R % 8 == 0 ? 3 : R % 4 == 0 ? 2 : R % 2 == 0 ? 1 : 0;
  s.tw_entries = s.tw_fold == 0 ? R : (R >> s.tw_fold) + 1;
  s.tw_shared = 1;
  // eight elements a thread where possible: the level kernels then fit 64
  // registers (two CTAs an SM) without spilling
  if (plan_with_E(R, 8, 512, s)) return true;
  return make_fft_plan(R, s);
}

// The swizzled column layout of a level (work_slot; kernels for the FP32
// levels' E = 8 and 16 schedules and the float-float forward levels' E = 8
// schedules of sub-FFTs in whole 16-point blocks): mask 15, else
// 0 (plain layout, no slot arithmetic).  Measured on the 4096 x 2048 FP32
// inverse levels of n = 2^24: both about 21 % faster (the first pass's 16-way
// store conflicts gone); the float-float forward levels gain less (0.7 % of a
// 2^24 decomposition); neutral on the uneven batch's lengths.
int level_swizzle(int R, int E) { return R % 16 == 0 && (E == 8 || E == 16) ? 15 : 0; }

int pick_tj(int R, int T, int count, size_t elem, size_t extra, int smem_limit) {
  for (int tj : {4, 3, 2, 1}) {
    if (count % tj) continue;
    if (tj * T > 512) continue;
    if ((size_t)tj * R * elem + extra + 1024 > (size_t)smem_limit) continue;
    return tj;
  }
  return 0;
}

// Nc = R1 R2 with R1, R2 <= 4096, as balanced as possible.
bool make_large_sched(int64_t n64, int smem_limit, LgSched& G) {
  if (n64 < 4 || n64 > (1 << 25) || !is_smooth(n64)) return false;
  memset(&G, 0, sizeof(G));
  FftSched& s = G.S;
  const int n = (int)n64;
  s.n = n;
  s.odd = n & 1;
  s.Nc = s.odd ? n : n / 2;
  s.P = s.odd ? (n + 1) / 2 : n / 2 + 1;
  s.Lmax = (n + 1) / 2;
  const int Nc = s.Nc;
  int best = 0;
  for (int d = 1; d <= 4096 && d <= Nc; d++) {
    if (Nc % d || Nc / d > 4096 || !is_smooth(d)) continue;
    const int e = Nc / d;
    if (!best || abs(d - e) < abs(best - Nc / best)) best = d;
  }
  if (!best) return false;
  G.R1 = best >= Nc / best ? best : Nc / best;
  G.R2 = Nc / G.R1;
  if (G.R2 < 2) return false;
  if (!make_sub_sched(G.R1, G.S1) || !make_sub_sched(G.R2, G.S2)) return false;
  const size_t t1 = tw_slots(G.S1) * sizeof(float2), t2 = tw_slots(G.S2) * sizeof(float2);
  G.TJ1 = pick_tj(G.R1, G.S1.T, G.R2, 8, t1, smem_limit);
  G.TJ2 = pick_tj(G.R2, G.S2.T, G.R1, 8, t2, smem_limit);
  G.F1 = G.S1;
  G.F2 = G.S2;
  G.S1.swz = level_swizzle(G.R1, G.S1.E);
  G.S2.swz = level_swizzle(G.R2, G.S2.E);
  G.F1.swz = G.F1.E == 8 ? level_swizzle(G.R1, 8) : 0;  // (float-float kernels: E = 8 only)
  G.F2.swz = G.F2.E == 8 ? level_swizzle(G.R2, 8) : 0;
  G.TJF1 = pick_tj(G.R1, G.F1.T, G.R2, 16, 0, smem_limit);
  G.TJF2 = pick_tj(G.R2, G.F2.T, G.R1, 16, 0, smem_limit);
  if (!G.TJ1 || !G.TJ2 || !G.TJF1 || !G.TJF2) return false;
  // the inter-level twiddle split: B the least power of two with B^2 >= Nc
  G.Bs = 0;
  while ((int64_t)1 << (2 * G.Bs) < Nc) G.Bs++;
  G.B = 1 << G.Bs;
  return true;
}

// One FP32 inverse level's schedule: sub-FFTs of R points with E elements a
// thread, tj of them per CTA.  false if it does not fit (threads, shared
// memory, tile count).
bool set_level(LgSched& G, int level, int E, int tj, int smem_limit) {
  const int R = level == 1 ? G.R1 : G.R2, count = level == 1 ? G.R2 : G.R1;
  FftSched sub = level == 1 ? G.S1 : G.S2;
  if (!plan_with_E(R, E, 512, sub)) return false;
  sub.ptw = nullptr;  // the per-pass table of the new radix sequence: large_pass_tables
  sub.swz = level_swizzle(R, E);
  if (tj < 1 || count % tj || tj * sub.T > 512) return false;
  if ((size_t)tj * (R + kLgColPad) * 8 + tw_slots(sub) * sizeof(float2) + 1024 > (size_t)smem_limit)
    return false;
  if (level == 1) {
    G.S1 = sub;
    G.TJ1 = tj;
  } else {
    G.S2 = sub;
    G.TJ2 = tj;
  }
  return true;
}

fif_status get_large(fif_plan_t p, int64_t n, LargeTables** out) {
  auto it = p->large.find(n);
  if (it != p->large.end()) {
    *out = &it->second;
    return FIF_OK;
  }
  LargeTables lt;
  if (!make_large_sched(n, p->smem_optin, lt.G)) return FIF_EUNSUPPORTED;
  LgSched& G = lt.G;
  {
    // m search: at most 4 CTAs per SM, at least 32 bins per thread
    const int want = (G.S.P + 32 * 256 - 1) / (32 * 256), cap = 4 * (p->num_sms > 0 ? p->num_sms : 1);
    G.sel_blocks = want < cap ? want : cap;
    if (G.sel_blocks > kSelBlocksMax) G.sel_blocks = kSelBlocksMax;
    if (G.sel_blocks < 1) G.sel_blocks = 1;
  }
  cudaError_t e = cudaSuccess;
  auto alloc = [&](size_t bytes) -> void* {
    void* ptr = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&ptr, bytes < 16 ? 16 : bytes);
    if (e == cudaSuccess) lt.allocs.push_back(ptr);
    return ptr;
  };
  const int n32 = (int)n, Nc = G.S.Nc, nhi = (Nc + G.B - 1) / G.B;
  float2* tw = (float2*)alloc(sizeof(float2) * n32);
  float2* twl = (float2*)alloc(sizeof(float2) * n32);
  double* s64 = (double*)alloc(sizeof(double) * (n32 / 2 + 1));
  float2* tw1 = (float2*)alloc(sizeof(float2) * G.R1);
  float2* tw1l = (float2*)alloc(sizeof(float2) * G.R1);
  double* d1 = (double*)alloc(sizeof(double) * (G.R1 / 2 + 1));
  float2* tw2 = (float2*)alloc(sizeof(float2) * G.R2);
  float2* tw2l = (float2*)alloc(sizeof(float2) * G.R2);
  double* d2 = (double*)alloc(sizeof(double) * (G.R2 / 2 + 1));
  float2* thi = (float2*)alloc(sizeof(float2) * nhi);
  float2* thil = (float2*)alloc(sizeof(float2) * nhi);
  float2* tlo = (float2*)alloc(sizeof(float2) * G.B);
  float2* tlol = (float2*)alloc(sizeof(float2) * G.B);
  float2* sff = (float2*)alloc(sizeof(float2) * (n32 / 2 + 1));
  float2* rff = (float2*)alloc(sizeof(float2) * (n32 / 2 + 1));
  if (e == cudaSuccess) e = build_twiddles(n32, tw, twl, s64, p->stream);
  if (e == cudaSuccess) e = build_twiddles(G.R1, tw1, tw1l, d1, p->stream);
  if (e == cudaSuccess) e = build_twiddles(G.R2, tw2, tw2l, d2, p->stream);
  G.S.tw = tw;
  G.S.tw_lo = twl;
  G.S.sin64 = s64;
  G.S.om64 = nullptr;  // shape window: each kernel points it at its signal's row
  G.S.om64_stride = 0;
  G.shape = p->d_shape;
  G.shape_len = (int)p->shape.size();
  G.S1.tw = G.F1.tw = tw1;
  G.S1.tw_lo = G.F1.tw_lo = tw1l;
  G.S2.tw = G.F2.tw = tw2;
  G.S2.tw_lo = G.F2.tw_lo = tw2l;
  G.thi = thi;
  G.thi_lo = thil;
  G.tlo = tlo;
  G.tlo_lo = tlol;
  G.sinff = sff;
  G.rcpff = rff;
  if (e == cudaSuccess) e = large_build_tables(G, thi, thil, tlo, tlol, sff, rff, p->stream);
  if (p->desc.precision == FIF_PREC_SPLIT_BF16) {
    // the split-BF16 variant: each FP32 inverse level whose sub-FFT takes an
    // E = 16 schedule with warp-aligned transforms runs its radix-16 passes on
    // the tensor cores
    for (int level = 1; level <= 2; level++) {
      for (int tj : {4, 3, 2, 1}) {
        LgSched t = G;
        if (!set_level(t, level, 16, tj, p->smem_optin)) continue;
        const FftSched& sub = level == 1 ? t.S1 : t.S2;
        bool r16 = false;
        for (int q = 0; q < sub.npass; q++) r16 |= sub.radix[q] == 16;
        if (!r16 || sub.T % 32) break;
        G = t;
        (level == 1 ? G.tc1 : G.tc2) = 1;
        break;
      }
    }
  } else {
    // a tuned (or loaded) schedule of the inverse levels replaces the rule's
    auto tv = p->large_sched.find(n);
    if (tv != p->large_sched.end()) {
      LgSched t = G;
      if (set_level(t, 1, tv->second[0], tv->second[1], p->smem_optin) &&
          set_level(t, 2, tv->second[2], tv->second[3], p->smem_optin))
        G = t;
    }
  }
  if (e == cudaSuccess) e = large_pass_tables(lt, G, p->stream);
  if (e == cudaSuccess) e = large_set_attrs(G);
  if (e != cudaSuccess) {
    for (void* a : lt.allocs) cudaFree(a);
    for (auto& pw : lt.ptw) cudaFree(pw.second);
    cudaGetLastError();
    return cuda_status(e);
  }
  auto res = p->large.emplace(n, lt);
  *out = &res.first->second;
  return FIF_OK;
}

void free_large_buffers(LargeBuffers& b) {
  for (void* a : b.allocs) cudaFree(a);
  b = LargeBuffers();
}

// Working arrays of one large class for nsig signals (grow-only, per length).
fif_status large_buffers(fif_plan_t p, const LgSched& G, int nsig, LargeBuffers** out,
                         bool single = false) {
  LargeBuffers& b = single ? p->large_single_bufs[G.S.n] : p->large_bufs[G.S.n];
  if (b.cap >= nsig) {
    *out = &b;
    return FIF_OK;
  }
  cudaStreamSynchronize(p->stream);
  free_large_buffers(b);
  const size_t Nc = (size_t)G.S.Nc, n = (size_t)G.S.n, P = (size_t)G.S.P, S = (size_t)nsig;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](size_t bytes) -> void* {
    void* ptr = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&ptr, bytes);
    if (e == cudaSuccess) b.allocs.push_back(ptr);
    return ptr;
  };
  b.za = (float4*)alloc(16 * Nc * S);
  b.zb = (float4*)alloc(16 * Nc * S);
  b.spec = (float2*)alloc(8 * (Nc + 1) * S);
  b.work = (float2*)alloc(8 * (Nc + 1) * S);
  b.work2 = (float2*)alloc(8 * (Nc + 1) * S);
  b.rem = (float*)alloc(4 * n * S);
  b.rem2 = (float*)alloc(4 * n * S);
  b.row = (float2*)alloc(8 * P * S);
  b.st = (int*)alloc(sizeof(int) * kLgStateWords * S);
  b.part = (unsigned char*)alloc((size_t)G.sel_blocks * kSelCand * kSelPartBytes * S);
  if (G.shape) b.om64 = (double*)alloc(sizeof(double) * P * S);
  b.d_sigs = (LgSig*)alloc(sizeof(LgSig) * S);
  if (e != cudaSuccess) {
    free_large_buffers(b);
    cudaGetLastError();
    return cuda_status(e);
  }
  b.n = G.S.n;
  b.cap = nsig;
  *out = &b;
  return FIF_OK;
}

// Fill the descriptors of idx[0..count) (one length) into b->d_sigs (blocking
// upload) and return the class.
fif_status upload_large_class(fif_plan_t p, const LgSched& G, LargeBuffers* b,
                              const int64_t* offsets, const int64_t* out_offsets,
                              const std::vector<int>& idx) {
  const int cnt = (int)idx.size();
  std::vector<LgSig> h(cnt);
  const size_t Nc = (size_t)G.S.Nc, P = (size_t)G.S.P;
  for (int q = 0; q < cnt; q++) {
    const int i = idx[q];
    LgSig& g = h[q];
    memset(&g, 0, sizeof(g));
    g.in_off = offsets ? offsets[i] : 0;
    g.out_off = out_offsets ? out_offsets[i] : 0;
    g.idx = i;
    g.za = b->za + Nc * q;
    g.zb = b->zb + Nc * q;
    g.spec = b->spec + (Nc + 1) * q;
    g.work = b->work + (Nc + 1) * q;
    g.work2 = b->work2 + (Nc + 1) * q;
    g.rem = b->rem + (size_t)G.S.n * q;
    g.rem2 = b->rem2 + (size_t)G.S.n * q;
    g.row = b->row + P * q;
    g.st = b->st + (size_t)kLgStateWords * q;
    g.part = b->part + (size_t)G.sel_blocks * kSelCand * kSelPartBytes * q;
    g.om64 = b->om64 ? b->om64 + P * q : nullptr;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_sigs, h.data(), sizeof(LgSig) * cnt,
                                  cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  return cuda_status(e);
}

// One signal of length n through the multi-pass path (fif_decompose).
fif_status run_large_single(fif_plan_t p, int64_t n, const float* signal, const Outputs& o) {
  LargeTables* lt = nullptr;
  fif_status s = get_large(p, n, &lt);
  if (s != FIF_OK) return s;
  LargeBuffers* b = nullptr;
  s = large_buffers(p, lt->G, 1, &b, true);
  if (s != FIF_OK) return s;
  std::vector<int> one(1, 0);
  s = upload_large_class(p, lt->G, b, nullptr, nullptr, one);
  if (s != FIF_OK) return s;
  cudaError_t e = cudaMemsetAsync(b->st, 0, sizeof(int) * kLgStateWords, p->stream);
  if (e == cudaSuccess) e = large_run(lt->G, b->d_sigs, 1, p->mp, signal, o, p->stream);
  return cuda_status(e);
}

// Tables, working arrays and descriptors of the large classes of a fresh
// layout.
fif_status prepare_large(fif_plan_t p, const int64_t* offsets, const int64_t* out_offsets,
                         const std::map<int64_t, std::vector<int>>& groups) {
  BatchLayout& l = p->layout;
  l.lcls.clear();
  for (const auto& kv : groups) {
    LargeTables* lt = nullptr;
    fif_status s = get_large(p, kv.first, &lt);
    if (s != FIF_OK) return s;
    const int cnt = (int)kv.second.size();
    if (cnt > 65535) return FIF_EUNSUPPORTED;
    LargeBuffers* b = nullptr;
    s = large_buffers(p, lt->G, cnt, &b);
    if (s != FIF_OK) return s;
    s = upload_large_class(p, lt->G, b, offsets, out_offsets, kv.second);
    if (s != FIF_OK) return s;
    l.lcls.push_back(BatchLayout::LargeCls{kv.first, cnt, lt, b});
  }
  return FIF_OK;
}

// Enqueue every class of the current layout; with more than one class each
// goes to its own branch stream (fork/join by events), so that independent
// lengths run side by side (and become parallel branches of a captured graph).
// Each length class runs on one of kBranches forked streams (parallel
// branches of the captured graph).  Classes are dealt longest first to the
// branch with the least estimated work (count * n log2 n, the multi-pass path
// weighted for its passes through global memory).
fif_status enqueue_batch(fif_plan_t p, const float* signals, const Outputs& o) {
  const BatchLayout& l = p->layout;
  const int nf = (int)l.classes.size(), ncls = nf + (int)l.lcls.size();
  const bool fork = ncls > 1;
  cudaError_t e = cudaSuccess;
  if (fork) e = cudaEventRecord(p->ev_fork, p->stream);
  struct Job {
    double cost;
    int cls;
  };
  std::vector<Job> jobs;
  for (int c = 0; c < ncls; c++) {
    const double n = c < nf ? (double)l.classes[c].n : (double)l.lcls[c - nf].n;
    const double cnt = c < nf ? (double)l.classes[c].count : (double)l.lcls[c - nf].count;
    jobs.push_back(Job{cnt * n * std::log2(n + 1.0) * (c < nf ? 1.0 : 3.0), c});
  }
  std::stable_sort(jobs.begin(), jobs.end(), [](const Job& a, const Job& b) { return a.cost > b.cost; });
  double load[fif_plan_s::kBranches] = {0.0};
  bool used[fif_plan_s::kBranches] = {false};
  for (const Job& jb : jobs) {
    if (e != cudaSuccess) break;
    cudaStream_t s = p->stream;
    if (fork) {
      int a = 0;
      for (int b = 1; b < fif_plan_s::kBranches; b++)
        if (load[b] < load[a]) a = b;
      load[a] += jb.cost;
      if (!used[a]) e = cudaStreamWaitEvent(p->aux[a], p->ev_fork, 0);
      used[a] = true;
      s = p->aux[a];
    }
    if (e != cudaSuccess) break;
    if (jb.cls < nf) {
      const auto& cl = l.classes[jb.cls];
      e = launch_fused(cl.E, l.d_sigs + cl.first, cl.count, l.d_scheds, cl.smem, cl.threads,
                       cl.grid, p->mp, signals, o, l.d_counters + jb.cls, s, cl.tc);
    } else {
      const auto& lc = l.lcls[jb.cls - nf];
      e = cudaMemsetAsync(lc.b->st, 0, sizeof(int) * kLgStateWords * (size_t)lc.count, s);
      if (e == cudaSuccess) e = large_run(lc.lt->G, lc.b->d_sigs, lc.count, p->mp, signals, o, s);
    }
  }
  if (fork) {
    for (int a = 0; a < fif_plan_s::kBranches && e == cudaSuccess; a++) {
      if (!used[a]) continue;
      e = cudaEventRecord(p->ev_join[a], p->aux[a]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->ev_join[a], 0);
    }
  }
  return cuda_status(e);
}

bool fits_fused(fif_plan_t p, int64_t n) {
  if (p->desc.flags & FIF_FORCE_MULTIPASS) return false;
  FftSched s;
  return make_sched(n, s, p->smem_optin) && fused_fits(s, p->smem_optin);
}

bool layout_matches(fif_plan_t p, const int64_t* offsets, const int64_t* out_offsets,
                    int64_t batch) {
  const BatchLayout& l = p->layout;
  return p->layout_valid && (int64_t)l.out_offsets.size() == batch &&
         std::equal(l.offsets.begin(), l.offsets.end(), offsets) &&
         std::equal(l.out_offsets.begin(), l.out_offsets.end(), out_offsets);
}

// ---- schedule autotuning helpers ---------------------------------------------------

// Fused schedules a length may use, the default first.
std::vector<FftSched> fused_candidates(const LengthTables& t) {
  std::vector<FftSched> out;
  FftSched first = t.sched;
  if (make_fft_plan(t.sched.Nc, first, true)) out.push_back(first);
  for (int E : {2, 3, 4, 6, 8, 9, 12, 16, 18, 24, 27}) {
    FftSched c = t.sched;
    if (!plan_with_E(t.sched.Nc, E, fused_max_threads(E), c, true)) continue;
    if (!out.empty() && c.E == out[0].E) continue;
    if (fused_blocks_per_sm(c.E, (int)fused_smem_bytes(c), sched_threads(c)) <= 0) continue;
    out.push_back(c);
  }
  return out;
}

void drop_layout(fif_plan_t p) {
  free_layout(p->layout);
  p->layout_valid = false;
}

}  // namespace

extern "C" {

const char* fif_status_string(fif_status s) {
  switch (s) {
    case FIF_OK: return "FIF_OK";
    case FIF_EINVAL: return "FIF_EINVAL: invalid argument";
    case FIF_ENOMEM: return "FIF_ENOMEM: device allocation failed";
    case FIF_ECUDA: return "FIF_ECUDA: CUDA runtime or launch error";
    case FIF_ETIMEOUT: return "FIF_ETIMEOUT: bounded device wait gave up";
    case FIF_EUNSUPPORTED: return "FIF_EUNSUPPORTED: request not implemented";
  }
  return "unknown fif_status";
}

int64_t fif_fused_max_n(void) {
  const int optin = device_smem_optin();
  if (optin <= 0) return 0;
  int64_t best = 0;
  for (int64_t p3 = 1; p3 <= (1 << 24); p3 *= 3) {
    for (int64_t n = p3; n <= (1 << 24); n *= 2) {
      FftSched s;
      if (n > best && make_sched(n, s, optin) && fused_fits(s, optin)) best = n;
    }
  }
  return best;
}

fif_status fif_plan_create(fif_plan_t* out, const fif_plan_desc* desc, void* cuda_stream) {
  if (!out) return FIF_EINVAL;
  *out = nullptr;
  fif_status st = validate_desc(desc);
  if (st != FIF_OK) return st;
  fif_plan_s* p = new (std::nothrow) fif_plan_s();
  if (!p) return FIF_ENOMEM;
  p->desc = *desc;
  if (desc->window == FIF_WIN_SHAPE) {
    p->shape.assign(desc->window_shape, desc->window_shape + desc->window_shape_len);
    p->desc.window_shape = p->shape.data();
  } else {
    p->desc.window_shape = nullptr;
    p->desc.window_shape_len = 0;
  }
  p->mp.nu = desc->nu;
  p->mp.delta = desc->delta;
  p->mp.delta2 = (float)(desc->delta * desc->delta);
  p->mp.mask_scale = desc->mask_scale;
  p->mp.max_inner = desc->max_inner;
  p->mp.max_imfs = desc->max_imfs;
  p->mp.force_L = (desc->flags & FIF_FORCE_L) ? 1 : 0;
  p->mp.apriori = (desc->flags & FIF_APRIORI_N0) ? 1 : 0;
  p->mp.peak_mask = (desc->flags & FIF_PEAK_MASK) ? 1 : 0;
  p->mp.threshold = desc->gamma > 0.0 ? 1 : 0;
  p->mp.gamma = desc->gamma;
  p->mp.log2_keep = desc->gamma > 0.0 ? (float)log2(1.0 - desc->gamma) : 0.f;
  p->stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) p->smem_optin = device_smem_optin();
  // scratch of the staged single-signal path, sized for max_n
  const int64_t n = desc->max_n;
  if (e == cudaSuccess) e = cudaMalloc(&p->scr.spec, sizeof(float2) * (size_t)(n / 2 + 2));
  if (e == cudaSuccess) e = cudaMalloc(&p->scr.work, sizeof(float2) * (size_t)(n + 2));
  if (e == cudaSuccess) e = cudaMalloc(&p->scr.rem, sizeof(float) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&p->scr.state, sizeof(int) * 16);
  if (e == cudaSuccess && !p->shape.empty()) {
    e = cudaMalloc(&p->d_shape, sizeof(double) * p->shape.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_shape, p->shape.data(), sizeof(double) * p->shape.size(),
                     cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    fif_plan_destroy(p);
    cudaGetLastError();
    return cuda_status(e);
  }
  for (int a = 0; a < fif_plan_s::kBranches && e == cudaSuccess; a++) {
    e = cudaStreamCreateWithFlags(&p->aux[a], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join[a], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    fif_plan_destroy(p);
    cudaGetLastError();
    return cuda_status(e);
  }
  p->scr_n = n;
  *out = p;
  return FIF_OK;
}

fif_status fif_plan_destroy(fif_plan_t p) {
  if (!p) return FIF_OK;
  cudaStreamSynchronize(p->stream);
  for (auto& kv : p->tables) {
    cudaFree(kv.second.tw);
    cudaFree(kv.second.tw_lo);
    cudaFree(kv.second.wtab);
    cudaFree(kv.second.sin64);
    cudaFree(kv.second.om64);
    cudaFree(kv.second.ltab);
    cudaFree(kv.second.gtab);
    for (auto& pw : kv.second.ptw) cudaFree(pw.second);
  }
  cudaFree(p->d_shape);
  free_layout(p->layout);
  for (auto& kv : p->large) {
    for (void* a : kv.second.allocs) cudaFree(a);
    for (auto& pw : kv.second.ptw) cudaFree(pw.second);
  }
  for (auto& kv : p->large_bufs) free_large_buffers(kv.second);
  cudaFree(p->scr.spec);
  cudaFree(p->scr.work);
  cudaFree(p->scr.rem);
  cudaFree(p->scr.state);
  cudaFree(p->h2d_buf);
  for (int a = 0; a < fif_plan_s::kBranches; a++) {
    if (p->aux[a]) cudaStreamSynchronize(p->aux[a]);
    if (p->aux[a]) cudaStreamDestroy(p->aux[a]);
    if (p->ev_join[a]) cudaEventDestroy(p->ev_join[a]);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  delete p;
  return FIF_OK;
}

fif_status fif_plan_set_stream(fif_plan_t p, void* cuda_stream) {
  if (!p) return FIF_EINVAL;
  p->stream = (cudaStream_t)cuda_stream;
  return FIF_OK;
}

fif_status fif_plan_prepare(fif_plan_t p, const int64_t* lengths, int64_t count) {
  if (!p || count < 0 || (count > 0 && !lengths)) return FIF_EINVAL;
  cudaGetLastError();
  for (int64_t i = 0; i < count; i++) {
    if (lengths[i] > p->desc.max_n || !is_smooth(lengths[i])) return FIF_EUNSUPPORTED;
    fif_status st;
    FftSched probe;
    if (fits_fused(p, lengths[i]) ||
        (p->d_shape && make_sched(lengths[i], probe, p->smem_optin) &&
         staged_fits(probe, p->smem_optin))) {
      LengthTables* t = nullptr;
      st = get_tables(p, lengths[i], &t);
    } else {
      LargeTables* lt = nullptr;
      st = get_large(p, lengths[i], &lt);
    }
    if (st != FIF_OK) return st;
  }
  return cuda_status(cudaStreamSynchronize(p->stream));
}

fif_status fif_decompose(fif_plan_t p, const float* signal, int64_t n, float* imfs, int32_t* m,
                         int32_t* mask_len, int32_t* n_imfs, int32_t* sig_status,
                         fif_imf_diag* diag) {
  if (!p || !signal || !imfs || !n_imfs || !sig_status) return FIF_EINVAL;
  cudaGetLastError();  // a pending error of earlier, unrelated work is not this call's
  if (p->desc.max_imfs > 0 && (!m || !mask_len)) return FIF_EINVAL;
  if (n < 4 || n > p->desc.max_n) return n < 4 ? FIF_EINVAL : FIF_EUNSUPPORTED;
  if (!is_smooth(n)) return FIF_EUNSUPPORTED;
  FftSched probe;
  if ((p->desc.flags & FIF_FORCE_MULTIPASS) || !make_sched(n, probe, p->smem_optin) ||
      !staged_fits(probe, p->smem_optin)) {
    Outputs o{imfs, m, mask_len, n_imfs, sig_status, diag};
    return run_large_single(p, n, signal, o);
  }
  LengthTables* t = nullptr;
  fif_status st = get_tables(p, n, &t);
  if (st != FIF_OK) return st;
  Outputs o{imfs, m, mask_len, n_imfs, sig_status, diag};
  return cuda_status(launch_staged(t->sched, nullptr, p->mp, signal, o, p->scr, p->stream));
}

static fif_status check_batch(fif_plan_t p, const float* signals, const int64_t* offsets,
                              int64_t batch, const float* imfs, const int64_t* out_offsets,
                              const int32_t* m, const int32_t* mask_len, const int32_t* n_imfs,
                              const int32_t* sig_status) {
  if (!p || batch < 0 || batch > (1LL << 30)) return FIF_EINVAL;
  if (batch == 0) return FIF_OK;
  if (!signals || !offsets || !imfs || !out_offsets || !n_imfs || !sig_status) return FIF_EINVAL;
  if (p->desc.max_imfs > 0 && (!m || !mask_len)) return FIF_EINVAL;
  if (offsets[0] != 0) return FIF_EINVAL;
  for (int64_t i = 0; i < batch; i++) {
    const int64_t n = offsets[i + 1] - offsets[i];
    if (n < 4 || out_offsets[i] < 0) return FIF_EINVAL;
    if (n > p->desc.max_n || !is_smooth(n)) return FIF_EUNSUPPORTED;
  }
  return FIF_OK;
}


fif_status fif_decompose_batch(fif_plan_t p, const float* signals, const int64_t* offsets,
                               int64_t batch, float* imfs, const int64_t* out_offsets, int32_t* m,
                               int32_t* mask_len, int32_t* n_imfs, int32_t* sig_status,
                               fif_imf_diag* diag) {
  fif_status st = check_batch(p, signals, offsets, batch, imfs, out_offsets, m, mask_len, n_imfs,
                              sig_status);
  if (st != FIF_OK || batch == 0) return st;
  cudaGetLastError();  // a pending error of earlier, unrelated work is not this call's
  if (!layout_matches(p, offsets, out_offsets, batch)) {
    std::vector<int> fused;
    std::map<int64_t, std::vector<int>> large;
    for (int64_t i = 0; i < batch; i++) {
      const int64_t n = offsets[i + 1] - offsets[i];
      if (fits_fused(p, n))
        fused.push_back((int)i);
      else
        large[n].push_back((int)i);
    }
    p->layout_valid = false;
    st = prepare_layout(p, offsets, out_offsets, batch, fused);
    if (st == FIF_OK) st = prepare_large(p, offsets, out_offsets, large);
    if (st != FIF_OK) {
      p->layout_valid = false;
      return st;
    }
  }
  Outputs o{imfs, m, mask_len, n_imfs, sig_status, diag};
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(p->stream, &cs);
  if (e != cudaSuccess) return cuda_status(e);
  if (cs != cudaStreamCaptureStatusNone) return enqueue_batch(p, signals, o);  // caller's graph
  // The legacy and per-thread default streams cannot be captured: enqueue directly.
  if (p->stream == nullptr || p->stream == cudaStreamLegacy || p->stream == cudaStreamPerThread)
    return enqueue_batch(p, signals, o);
  BatchLayout& l = p->layout;
  const void* key[8] = {signals, imfs, m, mask_len, n_imfs, sig_status, diag, (const void*)p->stream};
  if (!l.exec || !std::equal(key, key + 8, l.key)) {
    if (l.exec) {
      cudaGraphExecDestroy(l.exec);
      l.exec = nullptr;
    }
    e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return enqueue_batch(p, signals, o);
    }
    const fif_status es = enqueue_batch(p, signals, o);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(p->stream, &g);
    if (es != FIF_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return es != FIF_OK ? es : cuda_status(e);
    }
    e = cudaGraphInstantiate(&l.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      l.exec = nullptr;
      return cuda_status(e);
    }
    std::copy(key, key + 8, l.key);
  }
  return cuda_status(cudaGraphLaunch(l.exec, p->stream));
}

// Device address of a host buffer that kernels may read and write in place:
// page-locked memory mapped into the device's address space (cudaMallocHost,
// cudaHostAlloc, or cudaHostRegister with mapping).  nullptr for anything else.
static void* device_view(const void* h) {
  if (!h) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

fif_status fif_decompose_batch_host(fif_plan_t p, const float* signals, const int64_t* offsets,
                                    int64_t batch, float* imfs, const int64_t* out_offsets,
                                    int32_t* m, int32_t* mask_len, int32_t* n_imfs,
                                    int32_t* sig_status, fif_imf_diag* diag) {
  fif_status st = check_batch(p, signals, offsets, batch, imfs, out_offsets, m, mask_len, n_imfs,
                              sig_status);
  if (st != FIF_OK || batch == 0) return st;
  const int K1 = p->desc.max_imfs + 1;
  int64_t out_len = 0;
  for (int64_t i = 0; i < batch; i++)
    out_len = std::max(out_len, out_offsets[i] + (offsets[i + 1] - offsets[i]) * K1);
  const size_t in_b = sizeof(float) * (size_t)offsets[batch];
  const size_t out_b = sizeof(float) * (size_t)out_len;
  const size_t mi_b = sizeof(int32_t) * (size_t)batch * (size_t)p->desc.max_imfs;
  const size_t si_b = sizeof(int32_t) * (size_t)batch;
  const size_t dg_b = diag ? sizeof(fif_imf_diag) * (size_t)batch * (size_t)K1 : 0;
  // Mapped page-locked buffers are used in place: the kernels read the input
  // and write the outputs across the host link while they compute.  Other
  // buffers go through device staging with copies before and after.
  struct Buf {
    void* host;
    void* dev;  // in place, or the staging slot
    size_t bytes;
    bool in, out;
    bool staged;
  };
  Buf b[7] = {{(void*)signals, nullptr, in_b, true, false, false},
              {imfs, nullptr, out_b, false, true, false},
              {m, nullptr, mi_b, false, true, false},
              {mask_len, nullptr, mi_b, p->mp.force_L != 0, true, false},
              {n_imfs, nullptr, si_b, false, true, false},
              {sig_status, nullptr, si_b, false, true, false},
              {diag, nullptr, dg_b, false, true, false}};
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t need = 0;
  for (Buf& x : b) {
    if (!x.host || !x.bytes) continue;
    x.dev = device_view(x.host);
    x.staged = x.dev == nullptr;
    if (x.staged) need += al(x.bytes);
  }
  if (need > p->h2d_cap) {
    cudaFree(p->h2d_buf);
    p->h2d_buf = nullptr;
    p->h2d_cap = 0;
    cudaError_t e = cudaMalloc(&p->h2d_buf, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
    p->h2d_cap = need;
  }
  char* slot = (char*)p->h2d_buf;
  cudaStream_t s = p->stream;
  cudaError_t e = cudaSuccess;
  for (Buf& x : b) {
    if (!x.staged) continue;
    x.dev = slot;
    slot += al(x.bytes);
    if (x.in && e == cudaSuccess) e = cudaMemcpyAsync(x.dev, x.host, x.bytes, cudaMemcpyHostToDevice, s);
  }
  if (e != cudaSuccess) return cuda_status(e);
  st = fif_decompose_batch(p, (const float*)b[0].dev, offsets, batch, (float*)b[1].dev,
                           out_offsets, (int32_t*)b[2].dev, (int32_t*)b[3].dev,
                           (int32_t*)b[4].dev, (int32_t*)b[5].dev, (fif_imf_diag*)b[6].dev);
  if (st != FIF_OK) return st;
  for (Buf& x : b)
    if (x.staged && x.out && e == cudaSuccess)
      e = cudaMemcpyAsync(x.host, x.dev, x.bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e);
}

fif_status fif_plan_tune(fif_plan_t p, const float* signals, const int64_t* offsets, int64_t batch,
                         float* imfs, const int64_t* out_offsets, int32_t* m, int32_t* mask_len,
                         int32_t* n_imfs, int32_t* sig_status) {
  fif_status st = check_batch(p, signals, offsets, batch, imfs, out_offsets, m, mask_len, n_imfs,
                              sig_status);
  if (st != FIF_OK || batch == 0) return st;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(p->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return FIF_EINVAL;
  cudaGetLastError();
  // the split-BF16 variant's schedule is fixed (E = 16, radix-16 passes on the
  // tensor cores): nothing to tune, a plain batch call
  if (p->desc.precision == FIF_PREC_SPLIT_BF16)
    return fif_decompose_batch(p, signals, offsets, batch, imfs, out_offsets, m, mask_len, n_imfs,
                               sig_status, nullptr);
  std::vector<int> fused;
  std::map<int64_t, std::vector<FftSched>> cands;
  for (int64_t i = 0; i < batch; i++) {
    const int64_t n = offsets[i + 1] - offsets[i];
    if (!fits_fused(p, n)) continue;
    fused.push_back((int)i);
    if (!cands.count(n)) {
      LengthTables* t = nullptr;
      st = get_tables(p, n, &t);
      if (st != FIF_OK) return st;
      cands[n] = fused_candidates(*t);
    }
  }
  size_t rounds = 0;
  for (const auto& kv : cands) rounds = std::max(rounds, kv.second.size());
  std::map<int64_t, std::pair<float, int>> best;  // n -> (ms, E)
  Outputs o{imfs, m, mask_len, n_imfs, sig_status, nullptr};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (size_t r = 0; r < rounds && e == cudaSuccess && st == FIF_OK; r++) {
    // round r: every length takes its r-th candidate (or keeps its last one)
    for (const auto& kv : cands) {
      if (kv.second.empty()) continue;
      p->fused_E[kv.first] = kv.second[std::min(r, kv.second.size() - 1)].E;
    }
    drop_layout(p);
    st = prepare_layout(p, offsets, out_offsets, batch, fused, false);
    if (st != FIF_OK) break;
    const BatchLayout& l = p->layout;
    for (size_t c = 0; c < l.classes.size() && e == cudaSuccess; c++) {
      const auto& cl = l.classes[c];
      const auto& cv = cands[cl.n];
      if (r > 0 && r >= cv.size()) continue;  // nothing new for this length
      float best_ms = 0.f;
      for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {  // one warm-up, two timed
        e = cudaEventRecord(e0, p->stream);
        if (e == cudaSuccess)
          e = launch_fused(cl.E, l.d_sigs + cl.first, cl.count, l.d_scheds, cl.smem, cl.threads,
                           cl.grid, p->mp, signals, o, l.d_counters + c, p->stream, cl.tc);
        if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 1 || (rep == 2 && ms < best_ms)) best_ms = ms;
      }
      auto b = best.find(cl.n);
      if (e == cudaSuccess && (b == best.end() || best_ms < b->second.first))
        best[cl.n] = std::make_pair(best_ms, cl.E);
    }
  }
  for (const auto& kv : best) p->fused_E[kv.first] = kv.second.second;
  // multi-pass classes: the two FP32 inverse levels (the path's main cost, once
  // per IMF), one level at a time: the sub-FFT schedule (E) and the sub-FFTs a
  // CTA transforms (TJ), each candidate timed on a whole run of the class
  std::map<int64_t, std::vector<int>> large;
  for (int64_t i = 0; i < batch; i++) {
    const int64_t n = offsets[i + 1] - offsets[i];
    if (!fits_fused(p, n)) large[n].push_back((int)i);
  }
  if (e == cudaSuccess && st == FIF_OK && !large.empty()) {
    drop_layout(p);
    st = prepare_large(p, offsets, out_offsets, large);
    const BatchLayout& l = p->layout;
    for (size_t c = 0; st == FIF_OK && c < l.lcls.size() && e == cudaSuccess; c++) {
      const auto& lc = l.lcls[c];
      LgSched& G = lc.lt->G;
      auto run_ms = [&](LgSched t, float* ms) {
        cudaError_t r = large_pass_tables(*lc.lt, t, p->stream);
        if (r == cudaSuccess) r = large_set_attrs(t);
        float best_ms = 0.f;
        for (int rep = 0; rep < 2 && r == cudaSuccess; rep++) {  // one warm-up, one timed
          r = cudaMemsetAsync(lc.b->st, 0, sizeof(int) * kLgStateWords * (size_t)lc.count, p->stream);
          if (r == cudaSuccess) r = cudaEventRecord(e0, p->stream);
          if (r == cudaSuccess) r = large_run(t, lc.b->d_sigs, lc.count, p->mp, signals, o, p->stream);
          if (r == cudaSuccess) r = cudaEventRecord(e1, p->stream);
          if (r == cudaSuccess) r = cudaEventSynchronize(e1);
          if (r == cudaSuccess) r = cudaEventElapsedTime(&best_ms, e0, e1);
        }
        *ms = best_ms;
        return r;
      };
      for (int level = 1; level <= 2 && e == cudaSuccess; level++) {
        float best_ms = 0.f;
        e = run_ms(G, &best_ms);
        int bE = level == 1 ? G.S1.E : G.S2.E, btj = level == 1 ? G.TJ1 : G.TJ2;
        for (int E : {8, 16, 4, 12, 6, 24, 9, 18}) {
          for (int tj : {4, 3, 2, 1}) {
            if (e != cudaSuccess) break;
            LgSched t = G;
            if (!set_level(t, level, E, tj, p->smem_optin)) continue;
            if ((level == 1 ? t.S1.E : t.S2.E) == bE && (level == 1 ? t.TJ1 : t.TJ2) == btj) continue;
            float ms = 0.f;
            e = run_ms(t, &ms);
            if (e == cudaSuccess && ms < best_ms) best_ms = ms, bE = E, btj = tj;
          }
        }
        if (e == cudaSuccess) set_level(G, level, bE, btj, p->smem_optin);
      }
      if (e == cudaSuccess) e = large_pass_tables(*lc.lt, G, p->stream);
      if (e == cudaSuccess) e = large_set_attrs(G);
      if (e == cudaSuccess) p->large_sched[lc.n] = {G.S1.E, G.TJ1, G.S2.E, G.TJ2};
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  drop_layout(p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  if (st != FIF_OK) return st;
  return fif_decompose_batch(p, signals, offsets, batch, imfs, out_offsets, m, mask_len, n_imfs,
                             sig_status, nullptr);
}

fif_status fif_plan_batch_launches(fif_plan_t p, int64_t* launches) {
  if (!p || !launches) return FIF_EINVAL;
  *launches = 0;
  if (!p->layout_valid) return FIF_OK;
  int64_t c = (int64_t)p->layout.classes.size();  // one fused kernel a class
  for (const auto& lc : p->layout.lcls) c += large_launches(lc.count, p->mp, p->d_shape != nullptr);
  *launches = c;
  return FIF_OK;
}

fif_status fif_plan_get_schedule(fif_plan_t p, int64_t n, int32_t* E, int32_t* threads,
                                 int32_t* tuned) {
  if (!p || !E || !threads || !tuned) return FIF_EINVAL;
  if (n < 4 || n > p->desc.max_n || !is_smooth(n)) return FIF_EUNSUPPORTED;
  if (!fits_fused(p, n)) return FIF_EUNSUPPORTED;
  LengthTables* t = nullptr;
  const fif_status st = get_tables(p, n, &t);
  if (st != FIF_OK) return st;
  FftSched fs;
  fused_plan(p, t->sched, fs);
  *E = fs.E;
  *threads = sched_threads(fs);
  *tuned = p->fused_E.count(n) ? 1 : 0;
  return FIF_OK;
}

fif_status fif_plan_get_multipass_schedule(fif_plan_t p, int64_t n, int32_t* R1, int32_t* R2,
                                           int32_t* E1, int32_t* TJ1, int32_t* E2, int32_t* TJ2,
                                           int32_t* tuned) {
  if (!p || !R1 || !R2 || !E1 || !TJ1 || !E2 || !TJ2 || !tuned) return FIF_EINVAL;
  if (n < 4 || n > p->desc.max_n || !is_smooth(n)) return FIF_EUNSUPPORTED;
  if (fits_fused(p, n) && !(p->desc.flags & FIF_FORCE_MULTIPASS)) return FIF_EUNSUPPORTED;
  LargeTables* lt = nullptr;
  const fif_status st = get_large(p, n, &lt);
  if (st != FIF_OK) return st;
  const LgSched& G = lt->G;
  *R1 = G.R1, *R2 = G.R2, *E1 = G.S1.E, *TJ1 = G.TJ1, *E2 = G.S2.E, *TJ2 = G.TJ2;
  *tuned = p->large_sched.count(n) ? 1 : 0;
  return FIF_OK;
}

fif_status fif_plan_save_tuning(fif_plan_t p, const char* path) {
  if (!p || !path) return FIF_EINVAL;
  FILE* f = fopen(path, "w");
  if (!f) return FIF_EINVAL;
  for (const auto& kv : p->fused_E) fprintf(f, "%lld %d\n", (long long)kv.first, kv.second);
  for (const auto& kv : p->large_sched)
    fprintf(f, "%lld %d %d %d %d\n", (long long)kv.first, kv.second[0], kv.second[1], kv.second[2],
            kv.second[3]);
  return fclose(f) == 0 ? FIF_OK : FIF_EINVAL;
}

fif_status fif_plan_load_tuning(fif_plan_t p, const char* path) {
  if (!p || !path) return FIF_EINVAL;
  FILE* f = fopen(path, "r");
  if (!f) return FIF_EINVAL;
  std::map<int64_t, int> got;
  std::map<int64_t, std::array<int, 4>> got_large;
  char line[256];
  fif_status st = FIF_OK;
  while (fgets(line, sizeof line, f)) {
    long long n = 0;
    int E = 0, v[3] = {0, 0, 0};
    char extra = 0;
    const int k = sscanf(line, " %lld %d %d %d %d %c", &n, &E, &v[0], &v[1], &v[2], &extra);
    if (k == EOF || (k <= 0 && line[strspn(line, " \t\r\n")] == 0)) continue;  // blank
    if (k == 5) {  // a multi-pass length: E1 TJ1 E2 TJ2 of its inverse levels
      if (n < 4 || n > p->desc.max_n || !is_smooth(n) || fits_fused(p, n)) continue;
      LgSched G;
      if (!make_large_sched(n, p->smem_optin, G)) continue;
      if (!set_level(G, 1, E, v[0], p->smem_optin) || !set_level(G, 2, v[1], v[2], p->smem_optin))
        continue;
      got_large[(int64_t)n] = {E, v[0], v[1], v[2]};
      continue;
    }
    if (k != 2) {
      st = FIF_EINVAL;
      break;
    }
    if (n < 4 || n > p->desc.max_n || !is_smooth(n) || !fits_fused(p, n)) continue;
    FftSched base, c;
    if (!make_sched(n, base, p->smem_optin)) continue;
    c = base;
    if (!plan_with_E(base.Nc, E, fused_max_threads(E), c, true)) continue;
    got[(int64_t)n] = E;
  }
  fclose(f);
  if (st != FIF_OK) return st;
  for (const auto& kv : got) p->fused_E[kv.first] = kv.second;
  for (const auto& kv : got_large) {
    p->large_sched[kv.first] = kv.second;
    auto it = p->large.find(kv.first);  // tables already built: switch them over now
    if (it != p->large.end()) {
      LgSched t = it->second.G;
      if (set_level(t, 1, kv.second[0], kv.second[1], p->smem_optin) &&
          set_level(t, 2, kv.second[2], kv.second[3], p->smem_optin) &&
          large_pass_tables(it->second, t, p->stream) == cudaSuccess && large_set_attrs(t) == cudaSuccess)
        it->second.G = t;
    }
  }
  drop_layout(p);
  return FIF_OK;
}

}  // extern "C"
