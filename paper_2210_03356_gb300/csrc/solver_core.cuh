// Solve driver shared by the batch entry points and the server: CSR buffers,
// the per-matrix state, the precision stages and the round loop.
//
// A solve (Alg. 3.2.1) is a loop of rounds. The matrices of a batch live in
// stages, one per precision (FP32 for the first part of the mixed mode,
// FP64 otherwise); a stage holds its matrices as one block-diagonal CSR with
// global column indices, so every kernel launch serves all of them. Each
// round, each non-empty stage:
//   1. checks its iterates: T = X X and, per matrix, r = ||T - I||_F/sqrt(n),
//      x = ||X||_F/sqrt(n) and the budget (steps a2, a4);
//   2. per matrix: stops (r <= tol, step a7), diverges, runs out of updates,
//      moves from FP32 to FP64 (r < fp32_until, step a8), or updates;
//   3. for the updating matrices: Xbar = 1.5 X - 0.5 X T (step a3), the
//      threshold (step a5) and the filter with CSR compaction (step a6).
// A matrix that stops is copied out to its handle; the stage is rebuilt
// without it at the next round. Per-matrix control flow is exactly that of a
// lone solve, so every result is independent of the batch it ran in.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sign.h"
#include "common.cuh"
#include "kernels.h"

using namespace sgn;

namespace {

// Largest matrix order of the dense tensor-core path.
constexpr int64_t DENSE_MAX_N = 65536;
// Largest matrix order of NMF (its inverse is dense: three n x n FP64 blocks).
constexpr int64_t NMF_MAX_N = 32768;
// Buffers above this size are handed back as soon as they are not needed
// (between the update and the filter; when a stage empties).
constexpr size_t BIG_BUFFER = size_t(4) << 30;

// ------------------------------------------------------------------ CSR
template <typename T>
struct Csr {
  int64_t n = 0, nnz = 0;
  DevBuf rp, col, val;
  int64_t *d_rp() const { return rp.as<int64_t>(); }
  int32_t *d_col() const { return col.as<int32_t>(); }
  T *d_val() const { return val.as<T>(); }
  void ensure(int64_t rows, int64_t nz, cudaStream_t s) {
    n = rows;
    nnz = nz;
    rp.ensure(sizeof(int64_t) * size_t(rows + 1), s);
    col.ensure(sizeof(int32_t) * size_t(nz > 0 ? nz : 1), s);
    val.ensure(sizeof(T) * size_t(nz > 0 ? nz : 1), s);
  }
  void swap(Csr &o) {
    std::swap(n, o.n);
    std::swap(nnz, o.nnz);
    std::swap(rp.p, o.rp.p);
    std::swap(rp.cap, o.rp.cap);
    std::swap(rp.s, o.rp.s);
    std::swap(col.p, o.col.p);
    std::swap(col.cap, o.col.cap);
    std::swap(col.s, o.col.s);
    std::swap(val.p, o.val.p);
    std::swap(val.cap, o.val.cap);
    std::swap(val.s, o.val.s);
  }
};

}  // namespace

struct sign_ctx {
  int64_t n = 0, nnz = 0;
  cudaStream_t stream = nullptr;
  Csr<double> a;       // input copy
  Csr<double> result;  // last result
  bool has_result = false;
};

namespace {

template <typename T> constexpr int is_f32() { return sizeof(T) == 4; }

void sync(cudaStream_t s) { SGN_CUDA(cudaStreamSynchronize(s)); }

template <typename T>
void d2h(T *dst, const void *src, size_t count, cudaStream_t s) {
  SGN_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyDeviceToHost, s));
}
template <typename T>
void h2d(void *dst, const T *src, size_t count, cudaStream_t s) {
  SGN_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, s));
}

// Per-matrix bookkeeping of one solve call.
struct MatState {
  sign_t h = nullptr;
  sign_info *info = nullptr;
  int k = 0;            // updates done
  int status = -1;      // -1 running, else sign_status
  double resid = NAN;
  int trace_count = 0;
};

void trace_put(MatState &ms, int64_t nnz_x, int64_t nnz_t, double r, double x, int prec,
               double mults_t) {
  sign_info *in = ms.info;
  if (!in) return;
  int k = ms.trace_count;
  if (k >= in->cap) return;
  ms.trace_count++;
  if (in->nnz_x) in->nnz_x[k] = nnz_x;
  if (in->nnz_t) in->nnz_t[k] = nnz_t;
  if (in->resid_k) in->resid_k[k] = r;
  if (in->xnorm_k) in->xnorm_k[k] = x;
  if (in->beta_k) in->beta_k[k] = 0.0;
  if (in->tau_k) in->tau_k[k] = 0.0;
  if (in->fnorm_k) in->fnorm_k[k] = 0.0;
  if (in->nnz_bar) in->nnz_bar[k] = 0;
  if (in->prec_k) in->prec_k[k] = prec;
  if (in->mults_t) in->mults_t[k] = mults_t;
  if (in->mults_bar) in->mults_bar[k] = 0.0;
  if (in->nnz_that) in->nnz_that[k] = nnz_t;
}

// nnz of the filtered T the next update multiplies by (filter_t)
void trace_that(MatState &ms, int64_t nnz_that) {
  sign_info *in = ms.info;
  if (!in || !in->nnz_that || ms.trace_count == 0 || ms.trace_count > in->cap) return;
  in->nnz_that[ms.trace_count - 1] = nnz_that;
}

void trace_filter(MatState &ms, double beta, double tau, double fnorm, int64_t nnz_bar,
                  double mults_bar) {
  sign_info *in = ms.info;
  if (!in || ms.trace_count == 0 || ms.trace_count > in->cap) return;
  int k = ms.trace_count - 1;
  if (in->beta_k) in->beta_k[k] = beta;
  if (in->tau_k) in->tau_k[k] = tau;
  if (in->fnorm_k) in->fnorm_k[k] = fnorm;
  if (in->nnz_bar) in->nnz_bar[k] = nnz_bar;
  if (in->mults_bar) in->mults_bar[k] = mults_bar;
}

// A matrix waiting to enter a stage: its FP64 rows [row0, row0 + n) of a CSR
// it shares with the other matrices parked at the same time (the scaled
// inputs of one admission, or the iterates moving from FP32 to FP64 in one
// round); its columns start at col0 there.
struct Parked {
  int mat;
  std::shared_ptr<Csr<double>> owner;
  const int64_t *rp;
  const int32_t *col;
  const double *val;
  int64_t row0, n, col0, nnz;
};

// Output of a sparse product: row i occupies [rs[i], re[i]) of (col, val);
// rs is the exclusive scan of the row slot sizes, so gaps may follow a row.
template <typename T>
struct Slotted {
  int64_t n = 0, slots = 0;
  DevBuf rs, re, col, val;
  Rows rows() const { return Rows{rs.as<int64_t>(), re.as<int64_t>(), col.as<int32_t>()}; }
  T *d_val() const { return val.as<T>(); }
};

template <typename T>
Rows compact_rows(const Csr<T> &c) {
  return Rows{c.d_rp(), c.d_rp() + 1, c.d_col()};
}

// Band layout of one FP32 operand (see Band in kernels.h).
struct BandBuf {
  DevBuf fc, nf, span, pos, val, mask;
  int64_t total = 0;   // floats of the band (pos[n])
  bool filled = false;  // val and mask written for the current operand
  Band view() const {
    return Band{pos.as<int64_t>(), fc.as<int32_t>(), nf.as<int32_t>(), val.as<float>(),
                mask.as<unsigned>()};
  }
};

// Shared scratch of one solve call.
struct Work {
  DevBuf lo, len, ub, wlist, clist, counters, part, scan_tmp, eoff, sums, ms, active, sel,
      asm_blocks, asm_off, asm_lens, dropped, norm_work, norm, work, mults, cnt, nnzc, xblocks,
      dslot, dmem, dbufs, djobs, dscratch, dcount, derr;
  BandBuf bx, bt;  // bands of the iterate X and of T = X X (FP32 stage)
  DevBuf bandrow;  // rows of T written by the square's band tiles (1) or not (0)
  DevBuf n2v, n2y, n2z, n2part, n2zacc, n2xmax, n2ymax, n2nrm, x2;  // budget_norm
  int64_t sel_cap = 0;  // candidate room of the last threshold select
  DevBuf binfo;         // per row of a product's B: first/last column, length
  DevBuf nmf_int, nmf_dbl;  // NMF: permutation, pivot, singular flags; ||X^-1||
  bool bt_rows_done = false;  // the square's band tiles wrote their rows of T's band
};

// The matrices of one round on the dense path (FP32 stage): their slots,
// dense blocks and the batched product jobs.
struct DensePlan {
  std::vector<int> slot;          // per matrix of the stage: dense index or -1
  std::vector<DenseBuf> bufs;     // host copies of the device DenseBuf array (FP32 stage)
  std::vector<DenseBuf64> bufs64; // ... or of the DenseBuf64 array (FP64 stage)
  std::vector<int> mat;           // stage slot of each dense matrix
  int nd = 0, max_ld = 0;
  bool any() const { return nd > 0; }
};

// Page-locked host mirrors of the per-matrix values read back every round.
// Kept per host thread and grown only (cudaFreeHost would synchronize the
// device), so repeated solves reuse them.
struct HostMirror {
  void *p = nullptr;
  size_t cap = 0;
  MatScalars *ms = nullptr;
  int64_t *ex = nullptr, *nnz_t = nullptr, *nnz_bar = nullptr, *tot = nullptr;
  double *mults = nullptr, *dsum = nullptr;
  ExtractBlock *xb = nullptr;
  int *ctr = nullptr;  // the product's class counters
  void alloc(int nb) {
    size_t bytes = sizeof(MatScalars) * nb + sizeof(int64_t) * (4 * size_t(nb) + 8) +
                   sizeof(double) * 2 * size_t(nb) + sizeof(ExtractBlock) * nb +
                   sizeof(int) * RC_COUNTERS + 1024;
    if (bytes > cap) {
      if (p) cudaFreeHost(p);
      p = nullptr;
      SGN_CUDA(cudaMallocHost(&p, bytes));
      cap = bytes;
    }
    char *c = static_cast<char *>(p);
    auto take = [&](size_t b) {
      char *r = c;
      c += (b + 63) & ~size_t(63);
      return r;
    };
    ms = reinterpret_cast<MatScalars *>(take(sizeof(MatScalars) * nb));
    ex = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * (nb + 1)));
    nnz_t = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * nb));
    nnz_bar = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * nb));
    tot = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * 4));
    mults = reinterpret_cast<double *>(take(sizeof(double) * nb));
    dsum = reinterpret_cast<double *>(take(sizeof(double) * nb));
    xb = reinterpret_cast<ExtractBlock *>(take(sizeof(ExtractBlock) * nb));
    ctr = reinterpret_cast<int *>(take(sizeof(int) * RC_COUNTERS));
  }
  ~HostMirror() {
    if (p) cudaFreeHost(p);
  }
};

HostMirror &host_mirror() {
  static thread_local HostMirror hm;
  return hm;
}

template <typename T>
struct Stage {
  int prec = sizeof(T) == 4 ? 32 : 64;
  std::vector<int> mats;          // matrix ids, in row order
  std::vector<int> alive;         // 0 once a matrix has left (its rows are empty)
  std::vector<int64_t> moff;      // row offsets (host), size mats+1
  std::vector<int64_t> ex;        // entry offsets of X per matrix (host), size mats+1
  DevBuf d_moff, d_seg;
  Csr<T> X, Xh;                   // compact iterate and filtered update
  Slotted<T> Tm, Xb;              // X X and 1.5 X - 0.5 X T
  Csr<T> Th;                      // T after its filter (the filter_t variant)
  std::vector<std::unique_ptr<Parked>> incoming;  // matrices entering at the next round
};

// Pinned staging for the small host-to-device copies of the round loop.
// cudaMemcpyAsync from pageable memory first waits for the stream, so every
// such copy would stall the GPU; a copy from pinned memory is queued like a
// kernel. The bytes are copied into the arena at once (the caller may reuse
// its vector), and the arena is reused only after the stream has been
// synchronized, when every copy from it has completed.
struct Staging {
  char *p = nullptr;
  size_t cap = 0, used = 0;
  Staging() = default;
  Staging(const Staging &) = delete;
  Staging &operator=(const Staging &) = delete;
  ~Staging() {
    if (p) cudaFreeHost(p);
  }
  bool fits(size_t bytes) const { return used + ((bytes + 63) & ~size_t(63)) <= cap; }
  // the stream must be idle: nothing may still read the old arena
  void reserve(size_t bytes) {
    used = 0;
    if (bytes <= cap) return;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    SGN_CUDA(cudaMallocHost(reinterpret_cast<void **>(&p), bytes));
    cap = bytes;
  }
  void *put(const void *src, size_t bytes) {
    char *d = p + used;
    std::memcpy(d, src, bytes);
    used += (bytes + 63) & ~size_t(63);
    return d;
  }
};

struct Solver {
  cudaStream_t s;
  sign_opts o;
  std::vector<MatState> m;   // by matrix id
  std::vector<int> free_ids; // ids of collected matrices, reused by admit
  std::vector<int> retired;  // ids that stopped since the last collect()
  Work w;
  HostMirror &hm = host_mirror();
  Stage<float> s32;          // FP32 stage of the mixed mode
  Stage<double> s64;
  Staging stg;

  ~Solver() {
    if (stg.used) cudaStreamSynchronize(s);  // copies from the arena may be in flight
  }
  // Waits for the stream; the staging arena is free again afterwards.
  void wait() {
    prof_sync_point(s);
    sync(s);
    stg.used = 0;
  }
  // h2d from host memory of any kind, through the pinned arena.
  template <typename T>
  void put(void *dst, const T *src, size_t count) {
    const size_t bytes = sizeof(T) * count;
    if (bytes == 0) return;
    if (!stg.fits(bytes)) {
      wait();
      stg.reserve(std::max<size_t>(2 * stg.cap, std::max<size_t>(bytes + 64, size_t(1) << 18)));
    }
    SGN_CUDA(cudaMemcpyAsync(dst, stg.put(src, bytes), bytes, cudaMemcpyHostToDevice, s));
  }

  // ---------------------------------------------------------------- helpers
  void set_layout(std::vector<int64_t> &moff, const std::vector<int> &mats, DevBuf &d_moff,
                  DevBuf &d_seg) {
    moff.assign(mats.size() + 1, 0);
    for (size_t i = 0; i < mats.size(); ++i) moff[i + 1] = moff[i] + m[mats[i]].h->n;
    int64_t N = moff.back();
    d_moff.ensure(sizeof(int64_t) * moff.size(), s);
    put(d_moff.p, moff.data(), moff.size());
    d_seg.ensure(sizeof(int32_t) * size_t(N > 0 ? N : 1), s);
    launch_fill_seg(int(mats.size()), d_moff.as<int64_t>(), N, d_seg.as<int32_t>(), s);
  }

  // Assembles dst from blocks laid out one after another (block-diagonal).
  template <typename TD>
  void assemble(const std::vector<AsmBlock> &blocks, const std::vector<int64_t> &bnnz, Csr<TD> &dst) {
    int nb = int(blocks.size());
    std::vector<int64_t> boff(nb + 1, 0);
    int64_t nnz = 0;
    for (int b = 0; b < nb; ++b) {
      boff[b + 1] = boff[b] + blocks[b].nrows;
      nnz += bnnz[b];
    }
    int64_t N = boff[nb];
    dst.ensure(N, nnz, s);
    w.asm_blocks.ensure(sizeof(AsmBlock) * size_t(nb > 0 ? nb : 1), s);
    w.asm_off.ensure(sizeof(int64_t) * size_t(nb + 1), s);
    w.asm_lens.ensure(sizeof(int64_t) * size_t(N > 0 ? N : 1), s);
    w.scan_tmp.ensure(sizeof(int64_t) * size_t(scan_tmp_elems(N)), s);
    put(w.asm_blocks.p, blocks.data(), blocks.size());
    put(w.asm_off.p, boff.data(), boff.size());
    ProfScope ps(KC_ASSEMBLE, s, 0.0, double(nnz) * (8.0 + 4.0 + sizeof(TD)) + 16.0 * double(N));
    launch_assemble_rows(nb, w.asm_blocks.as<AsmBlock>(), w.asm_off.as<int64_t>(), N,
                         w.asm_lens.as<int64_t>(), dst.d_rp(), w.scan_tmp.as<int64_t>(), s);
    launch_assemble_vals(nb, w.asm_blocks.as<AsmBlock>(), w.asm_off.as<int64_t>(), N, dst.d_rp(),
                         dst.d_col(), dst.val.p, is_f32<TD>(), s);
  }

  // the band tiles' multiply-adds, a double after the class counters
  double *band_work_dev() {
    return reinterpret_cast<double *>(w.counters.as<char>() + sizeof(int) * RC_COUNTERS);
  }

  // ---------------------------------------------------------------- product
  // C = A B for a stage. Enqueues everything; on return C is allocated and the
  // product queued, hm.mults holds the per-matrix multiply-adds (synced) and
  // w.nnzc the per-matrix nnz of C (device, read with the next sync).
  template <typename T>
  void product(Stage<T> &st, const Rows &A, const T *aval, int64_t nnzA, const Rows &B,
               const T *bval, int64_t nnzB, int mode, Slotted<T> &C, const int *active,
               const DensePlan *dp = nullptr, bool b_is_square_t = true) {
    int64_t N = int64_t(st.moff.back());
    int nb = int(st.mats.size());
    w.lo.ensure(sizeof(int32_t) * size_t(N), s);
    w.len.ensure(sizeof(int32_t) * size_t(N), s);
    w.ub.ensure(sizeof(int64_t) * size_t(N), s);
    w.wlist.ensure(sizeof(int32_t) * size_t(RC_N) * size_t(N), s);
    w.work.ensure(sizeof(double) * size_t(N), s);
    w.mults.ensure(sizeof(double) * size_t(nb), s);
    w.nnzc.ensure(sizeof(int64_t) * size_t(nb), s);
    w.counters.ensure(sizeof(int) * RC_COUNTERS + sizeof(double), s);  // + band multiply-adds
    w.scan_tmp.ensure(sizeof(int64_t) * size_t(scan_tmp_elems(N)), s);
    SGN_CUDA(cudaMemsetAsync(w.counters.p, 0, sizeof(int) * RC_COUNTERS + sizeof(double), s));
    // band tiles (FP32): in SQUARE the bands of X (both operands) and of T
    // (the output, for the update) are laid out here, their sizes read with
    // the slot total below; the band tiles write the rows of T's band they
    // compute, and the update fills in the other rows of T it needs
    const bool band = sizeof(T) == 4 && o.fp32_band;
    {
      ProfScope ps(KC_BOUNDS, s);
      if (band && mode == MODE_SQUARE) w.bandrow.ensure(size_t(N > 0 ? N : 1), s);
      // schedule: FP64 rows by lane use (or all on 32 lanes), FP32 rows in pairs (or one per warp)
      const int groups = sizeof(T) == 8 ? (o.group_margin < 0.0 ? 0 : 1) : (o.pair_rows ? 2 : 0);
      launch_bounds(N, A, B, st.d_seg.template as<int32_t>(), active, mode, groups,
                    float(o.group_margin), band ? 1 : 0, float(o.band_min_eff),
                    dp && dp->any() ? w.dslot.as<int>() : nullptr,
                    st.d_moff.template as<int64_t>(), w.lo.as<int32_t>(),
                    w.len.as<int32_t>(), w.ub.as<int64_t>(), w.wlist.as<int32_t>(),
                    w.counters.as<int>(), w.work.as<double>(), band_work_dev(),
                    band && mode == MODE_SQUARE ? w.bandrow.as<unsigned char>() : nullptr,
                    static_cast<int4 *>(w.binfo.ensure(sizeof(int4) * size_t(N > 0 ? N : 1), s)),
                    s);
      launch_seg_reduce(nb, st.d_moff.template as<int64_t>(), w.work.as<double>(), 1,
                        w.mults.as<double>(), s);
      if (band) {
        if (mode == MODE_SQUARE) {
          for (BandBuf *b : {&w.bx, &w.bt}) {
            b->filled = false;
            b->fc.ensure(sizeof(int32_t) * size_t(N), s);
            b->nf.ensure(sizeof(int32_t) * size_t(N), s);
            b->span.ensure(sizeof(int64_t) * size_t(N), s);
            b->pos.ensure(sizeof(int64_t) * size_t(N + 1), s);
          }
          w.bt_rows_done = false;
          launch_band_spans(N, B, w.bx.fc.as<int32_t>(), w.bx.nf.as<int32_t>(),
                            w.bx.span.as<int64_t>(), s);
          launch_scan(N, w.bx.span.as<int64_t>(), w.bx.pos.as<int64_t>(),
                      w.scan_tmp.as<int64_t>(), s);
          launch_band_spans_range(N, w.lo.as<int32_t>(), w.len.as<int32_t>(),
                                  w.bt.fc.as<int32_t>(), w.bt.nf.as<int32_t>(),
                                  w.bt.span.as<int64_t>(), s);
          launch_scan(N, w.bt.span.as<int64_t>(), w.bt.pos.as<int64_t>(),
                      w.scan_tmp.as<int64_t>(), s);
          d2h(hm.tot + 1, w.bx.pos.as<int64_t>() + N, 1, s);
          d2h(hm.tot + 2, w.bt.pos.as<int64_t>() + N, 1, s);
        } else if (!b_is_square_t) {  // B is not the square's T: its own layout
          w.bt.filled = false;
          w.bt_rows_done = false;
          w.bt.fc.ensure(sizeof(int32_t) * size_t(N), s);
          w.bt.nf.ensure(sizeof(int32_t) * size_t(N), s);
          w.bt.span.ensure(sizeof(int64_t) * size_t(N), s);
          w.bt.pos.ensure(sizeof(int64_t) * size_t(N + 1), s);
          launch_band_spans(N, B, w.bt.fc.as<int32_t>(), w.bt.nf.as<int32_t>(),
                            w.bt.span.as<int64_t>(), s);
          launch_scan(N, w.bt.span.as<int64_t>(), w.bt.pos.as<int64_t>(),
                      w.scan_tmp.as<int64_t>(), s);
          d2h(hm.tot + 2, w.bt.pos.as<int64_t>() + N, 1, s);
        }
        d2h(hm.ctr, w.counters.p, RC_COUNTERS, s);
        d2h(hm.dsum, band_work_dev(), 1, s);
      }
    }
    C.n = N;
    C.rs.ensure(sizeof(int64_t) * size_t(N + 1), s);
    C.re.ensure(sizeof(int64_t) * size_t(N > 0 ? N : 1), s);
    {
      ProfScope ps(KC_SCAN, s);
      launch_scan(N, w.ub.as<int64_t>(), C.rs.template as<int64_t>(), w.scan_tmp.as<int64_t>(), s);
    }
    d2h(hm.tot, C.rs.template as<int64_t>() + N, 1, s);
    d2h(hm.mults, w.mults.p, size_t(nb), s);
    wait();
    int64_t slots = hm.tot[0];
    const bool band_tiles = band && hm.ctr[RC_BAND] > 0;
    if (band && mode == MODE_SQUARE) {
      w.bx.total = hm.tot[1];
      w.bt.total = hm.tot[2];
    } else if (band && !b_is_square_t) {
      w.bt.total = hm.tot[2];
    }
    if (band_tiles) {
      auto alloc = [&](BandBuf &b) {
        b.val.ensure(sizeof(float) * size_t(b.total + 4), s);
        b.mask.ensure(sizeof(unsigned) * size_t(b.total / 2 + 4), s);
      };
      // fills a band from its CSR rows (skipping the rows the band tiles wrote)
      auto fill = [&](BandBuf &b, const Rows &R, const T *v, const unsigned char *skip) {
        if (b.filled) return;
        alloc(b);
        launch_band_fill(N, R, reinterpret_cast<const float *>(v), b.pos.as<int64_t>(),
                         b.fc.as<int32_t>(), b.nf.as<int32_t>(), skip, b.val.as<float>(),
                         b.mask.as<unsigned>(), s);
        b.filled = true;
      };
      ProfScope ps(KC_BAND_LAYOUT, s, 0.0,
                   mode == MODE_SQUARE || !w.bt.filled
                       ? double(nnzB) * 8.0 + double(mode == MODE_SQUARE ? w.bx.total
                                                                         : w.bt.total) * 6.0
                       : 0.0);
      if (mode == MODE_SQUARE) {
        fill(w.bx, B, bval, nullptr);  // B = A = X
        alloc(w.bt);                    // written by the band tiles below
      } else {
        fill(w.bx, A, aval, nullptr);
        fill(w.bt, B, bval, w.bt_rows_done ? w.bandrow.as<unsigned char>() : nullptr);
      }
    }
    C.slots = slots;
    C.col.ensure(sizeof(int32_t) * size_t(slots > 0 ? slots : 1), s);
    C.val.ensure(sizeof(T) * size_t(slots > 0 ? slots : 1), s);
    if (mode == MODE_SQUARE) w.part.ensure(sizeof(double) * size_t(2 * N), s);
    double fl = 0.0;
    for (int i = 0; i < nb; ++i) fl += 2.0 * hm.mults[i];
    const double fl_band = band_tiles ? 2.0 * hm.dsum[0] : 0.0;  // the band tiles' share
    double per = 4.0 + sizeof(T);
    // algorithmic bytes: A and B read once, C written once (its size is known
    // after the launch; the slot total bounds it and is used here)
    double by = per * double(nnzA + (mode == MODE_UPDATE ? nnzB : 0) + slots) +
                8.0 * double(N + 1) * (mode == MODE_UPDATE ? 3.0 : 2.0) +
                (mode == MODE_SQUARE ? 16.0 * double(N) : 0.0);
    int cls = mode == MODE_SQUARE ? (sizeof(T) == 8 ? KC_NUM_SQUARE_F64 : KC_NUM_SQUARE_F32)
                                  : (sizeof(T) == 8 ? KC_NUM_UPDATE_F64 : KC_NUM_UPDATE_F32);
    {
      // bytes: the row-wise class keeps the whole product's algorithmic bytes
      ProfScope ps(cls, s, fl - fl_band, by);
      launch_numeric<T>(N, A, aval, B, bval, mode, w.lo.as<int32_t>(), w.len.as<int32_t>(),
                        w.wlist.as<int32_t>(), w.counters.as<int>(), C.rs.template as<int64_t>(),
                        C.re.template as<int64_t>(), C.col.template as<int32_t>(), C.d_val(),
                        mode == MODE_SQUARE ? w.part.as<double>() : nullptr, s);
    }
    if (band_tiles) {
      ProfScope ps(mode == MODE_SQUARE ? KC_BAND_SQUARE : KC_BAND_UPDATE, s, fl_band, 0.0);
      BandOut tout;
      if (mode == MODE_SQUARE) {
        tout = BandOut{w.bt.pos.as<int64_t>(), w.bt.fc.as<int32_t>(), w.bt.nf.as<int32_t>(),
                       w.bt.val.as<float>(), w.bt.mask.as<unsigned>()};
        w.bt_rows_done = true;  // the rows of bandrow; the update fills the rest
      }
      launch_band_product(N, mode, A, reinterpret_cast<const float *>(aval), w.bx.view(),
                          mode == MODE_SQUARE ? w.bx.view() : w.bt.view(), tout,
                          w.lo.as<int32_t>(), w.len.as<int32_t>(), w.wlist.as<int32_t>(),
                          w.counters.as<int>(), C.rs.template as<int64_t>(),
                          C.re.template as<int64_t>(), C.col.template as<int32_t>(),
                          reinterpret_cast<float *>(C.val.p),
                          mode == MODE_SQUARE ? w.part.as<double>() : nullptr, s);
    }
    if (dp && dp->any()) dense_step(st, mode, C, active, *dp);
    launch_seg_count(nb, st.d_moff.template as<int64_t>(), C.rs.template as<int64_t>(),
                     C.re.template as<int64_t>(), w.nnzc.as<int64_t>(), s);
  }

  // ---------------------------------------------------------------- dense path (a9)
  // Chooses the matrices of a stage whose iterate has filled in (density >=
  // dense_frac, n <= DENSE_MAX_N; in the FP64 stage also n >= dense64_min_n)
  // and lays out their dense blocks. A matrix whose blocks would not fit in
  // the device memory left (beside what the blocks of the last plan hold)
  // stays on the sparse path.
  template <typename T>
  DensePlan plan_dense(Stage<T> &st) {
    DensePlan dp;
    int nb = int(st.mats.size());
    dp.slot.assign(nb, -1);
    if (!(o.dense_frac <= 1.0) || o.filter == SIGN_FILTER_NONE || o.filter_t ||
        o.method == SIGN_METHOD_NMF)
      return dp;
    constexpr bool f32 = sizeof(T) == 4;
    size_t total = 0;  // bytes
    auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    // FP32: X, X^T, T^T split hi/lo and P; FP64: X, T^T, P and one K block's
    // digit planes and row exponents of the two operands
    auto bytes_of = [&](size_t ld) {
      return f32 ? 7 * 4 * ld * ld
                 : 3 * r256(8 * ld * ld) + 2 * r256(f64x_digits_bytes(int(ld), f64x_kd(int(ld)))) +
                       2 * r256(4 * ld);
    };
    size_t room = 0;
    bool room_known = false;
    for (int i = 0; i < nb; ++i) {
      if (!st.alive[i]) continue;
      int64_t n = st.moff[i + 1] - st.moff[i];
      int64_t nnz = st.ex[i + 1] - st.ex[i];
      // up to n = 65536: seven FP32 blocks (120 GB) in the FP32 stage; three
      // FP64 blocks and one K block's digit planes (112 GB) in the FP64 stage
      if (n > DENSE_MAX_N || double(nnz) < o.dense_frac * double(n) * double(n)) continue;
      if (!f32 && n < o.dense64_min_n) continue;  // too small to repay 36 passes per tile
      int ld = f32 ? int((n + 3) / 4 * 4) : int((n + 7) / 8 * 8);
      auto measure = [&] {  // free memory and the last plan's blocks, less headroom
        size_t fr = 0, tot = 0;
        SGN_CUDA(cudaMemGetInfo(&fr, &tot));
        const size_t have = fr + w.dmem.cap, keep = size_t(8) << 30;
        room = have > keep ? have - keep : 0;
      };
      if (!room_known) {
        measure();
        room_known = true;
      }
      if (total + bytes_of(size_t(ld)) > room && bytes_of(size_t(ld)) > BIG_BUFFER) {
        // memory kept for reuse (this thread's parked blocks, the pool's
        // free memory) goes back to the device before the path is refused
        block_cache_flush();
        SGN_CUDA(cudaDeviceSynchronize());
        SGN_CUDA(cudaMemPoolTrimTo(lib_pool(), 0));
        measure();
      }
      if (total + bytes_of(size_t(ld)) > room) continue;
      dp.slot[i] = dp.nd++;
      dp.mat.push_back(i);
      if (f32) {
        DenseBuf b = {};
        b.n = int(n);
        b.ld = ld;
        dp.bufs.push_back(b);
      } else {
        DenseBuf64 b = {};
        b.n = int(n);
        b.ld = ld;
        dp.bufs64.push_back(b);
      }
      dp.max_ld = std::max(dp.max_ld, ld);
      total += bytes_of(size_t(ld));
    }
    if (!dp.nd) return dp;
    unsigned char *mem = static_cast<unsigned char *>(w.dmem.ensure(total, s));
    size_t off = 0;
    if (f32) {
      for (DenseBuf &b : dp.bufs) {
        size_t blk = size_t(b.ld) * size_t(b.ld);
        float *base = reinterpret_cast<float *>(mem + off);
        b.X_hi = base;
        b.X_lo = base + blk;
        b.XT_hi = base + 2 * blk;
        b.XT_lo = base + 3 * blk;
        b.TT_hi = base + 4 * blk;
        b.TT_lo = base + 5 * blk;
        b.P = base + 6 * blk;
        off += bytes_of(size_t(b.ld));
      }
    } else {
      for (DenseBuf64 &b : dp.bufs64) {
        const size_t ld = size_t(b.ld), fb = r256(8 * ld * ld);
        b.kd = f64x_kd(b.ld);
        const size_t db = r256(f64x_digits_bytes(b.ld, b.kd)), eb = r256(4 * ld);
        unsigned char *p = mem + off;
        b.X = reinterpret_cast<double *>(p);
        b.TT = reinterpret_cast<double *>(p + fb);
        b.P = reinterpret_cast<double *>(p + 2 * fb);
        p += 3 * fb;
        b.dA = reinterpret_cast<uint16_t *>(p);
        b.dB = reinterpret_cast<uint16_t *>(p + db);
        p += 2 * db;
        b.eA = reinterpret_cast<int *>(p);
        b.eB = reinterpret_cast<int *>(p + eb);
        off += bytes_of(ld);
      }
    }
    w.dslot.ensure(sizeof(int) * size_t(nb), s);
    put(w.dslot.p, dp.slot.data(), size_t(nb));
    if (f32) {
      w.dbufs.ensure(sizeof(DenseBuf) * size_t(dp.nd), s);
      put(w.dbufs.p, dp.bufs.data(), size_t(dp.nd));
    } else {
      w.dbufs.ensure(sizeof(DenseBuf64) * size_t(dp.nd), s);
      put(w.dbufs.p, dp.bufs64.data(), size_t(dp.nd));
    }
    w.dcount.ensure(sizeof(unsigned long long) * size_t(dp.nd), s);
    w.derr.ensure(sizeof(int), s);
    SGN_CUDA(cudaMemsetAsync(w.derr.p, 0, sizeof(int), s));
    return dp;
  }

  // The dense steps of a product: SQUARE densifies X and forms T = X X and the
  // residual partials; UPDATE forms P = X T and emits 1.5 X - 0.5 P.
  template <typename T>
  void dense_step(Stage<T> &st, int mode, Slotted<T> &C, const int *active, const DensePlan &dp) {
    if constexpr (sizeof(T) == 4) {
      int64_t N = st.moff.back();
      std::vector<DenseJob> jobs;
      double fl = 0.0;
      for (const DenseBuf &b : dp.bufs) {
        if (mode == MODE_SQUARE)  // T^T = X^T X^T: C = A Bt^T with A = X^T, Bt = X
          jobs.push_back(DenseJob{b.ld, b.ld, b.ld, b.XT_hi, b.XT_lo, b.ld, b.X_hi, b.X_lo, b.ld,
                                  b.TT_hi, b.TT_lo, b.ld});
        else  // P = X T as C = A Bt^T with A = X, Bt = T^T
          jobs.push_back(DenseJob{b.ld, b.ld, b.ld, b.X_hi, b.X_lo, b.ld, b.TT_hi, b.TT_lo, b.ld,
                                  b.P, nullptr, b.ld});
        fl += 3.0 * 2.0 * double(b.ld) * double(b.ld) * double(b.ld);
      }
      w.djobs.ensure(sizeof(DenseJob) * jobs.size(), s);
      w.dscratch.ensure(dense_jobs_scratch_bytes(int(jobs.size())), s);
      const DenseBuf *bufs = w.dbufs.as<DenseBuf>();
      if (mode == MODE_SQUARE) {
        size_t total = 0;
        for (const DenseBuf &b : dp.bufs) total += 7 * size_t(b.ld) * size_t(b.ld);
        SGN_CUDA(cudaMemsetAsync(w.dmem.p, 0, sizeof(float) * total, s));
        launch_densify(N, st.d_seg.template as<int32_t>(), w.dslot.as<int>(),
                       st.d_moff.template as<int64_t>(), st.X.d_rp(), st.X.d_col(),
                       reinterpret_cast<const float *>(st.X.val.p), bufs, s);
      }
      {
        ProfScope ps(KC_DENSE, s, fl, 0.0);
        launch_dense_jobs(int(jobs.size()), jobs.data(), w.djobs.as<DenseJob>(), w.dscratch.p,
                          w.derr.as<int>(), s);
      }
      if (mode == MODE_SQUARE) {
        SGN_CUDA(cudaMemsetAsync(w.dcount.p, 0, sizeof(unsigned long long) * size_t(dp.nd), s));
        launch_dense_resid(N, st.d_seg.template as<int32_t>(), w.dslot.as<int>(),
                           st.d_moff.template as<int64_t>(), bufs, w.part.as<double>(),
                           w.dcount.as<unsigned long long>(), s);
      } else {
        launch_dense_emit(N, st.d_seg.template as<int32_t>(), w.dslot.as<int>(),
                          st.d_moff.template as<int64_t>(), active, bufs,
                          C.rs.template as<int64_t>(), C.re.template as<int64_t>(),
                          C.col.template as<int32_t>(), reinterpret_cast<float *>(C.val.p), s);
      }
    } else {
      int64_t N = st.moff.back();
      const DenseBuf64 *bufs = w.dbufs.as<DenseBuf64>();
      if (mode == MODE_SQUARE) {
        for (const DenseBuf64 &b : dp.bufs64)
          SGN_CUDA(cudaMemsetAsync(b.X, 0, sizeof(double) * size_t(b.ld) * size_t(b.ld), s));
        launch_densify64(N, st.d_seg.template as<int32_t>(), w.dslot.as<int>(),
                         st.d_moff.template as<int64_t>(), st.X.d_rp(), st.X.d_col(),
                         reinterpret_cast<const double *>(st.X.val.p), bufs, s);
      }
      // K blocks of F64X_MAX_K: every block's digits are cut just before its
      // product, which adds into C (SQUARE: C = T^T = X^T X^T as A Bt^T with
      // A = X^T, read transposed from X, and Bt = X; UPDATE: C = P = X T with
      // A = X and Bt = T^T)
      w.djobs.ensure(sizeof(SliceJob) * size_t(dp.nd), s);
      w.dscratch.ensure(slice_jobs_scratch_bytes(dp.nd), s);
      std::vector<SliceJob> jobs;
      for (int64_t k0 = 0; k0 < dp.max_ld; k0 += F64X_MAX_K) {
        jobs.clear();
        double fl = 0.0;
        for (const DenseBuf64 &b : dp.bufs64) {
          if (k0 >= b.ld) continue;
          const int K = int(std::min<int64_t>(F64X_MAX_K, b.ld - k0));
          const size_t ld = size_t(b.ld);
          if (mode == MODE_SQUARE) {
            launch_slices(b.ld, K, b.X + size_t(k0) * ld, b.ld, 1, b.dA, b.kd, b.eA, s);
            launch_slices(b.ld, K, b.X + size_t(k0), b.ld, 0, b.dB, b.kd, b.eB, s);
            jobs.push_back(SliceJob{b.ld, b.ld, K, b.dA, b.kd, b.dB, b.kd, b.eA, b.eB, b.TT, b.ld,
                                    k0 > 0 ? 1 : 0});
          } else {
            launch_slices(b.ld, K, b.X + size_t(k0), b.ld, 0, b.dA, b.kd, b.eA, s);
            launch_slices(b.ld, K, b.TT + size_t(k0), b.ld, 0, b.dB, b.kd, b.eB, s);
            jobs.push_back(SliceJob{b.ld, b.ld, K, b.dA, b.kd, b.dB, b.kd, b.eA, b.eB, b.P, b.ld,
                                    k0 > 0 ? 1 : 0});
          }
          fl += 2.0 * f64x_pairs() * double(b.ld) * double(b.ld) * double(K);
        }
        ProfScope ps(KC_DENSE64, s, fl, 0.0);
        launch_slice_jobs(int(jobs.size()), jobs.data(), w.djobs.as<SliceJob>(), w.dscratch.p,
                          w.derr.as<int>(), s);
      }
      if (mode == MODE_SQUARE) {
        SGN_CUDA(cudaMemsetAsync(w.dcount.p, 0, sizeof(unsigned long long) * size_t(dp.nd), s));
        launch_dense_resid64(N, st.d_seg.template as<int32_t>(), w.dslot.as<int>(),
                             st.d_moff.template as<int64_t>(), bufs, w.part.as<double>(),
                             w.dcount.as<unsigned long long>(), s);
      } else {
        launch_dense_emit64(N, st.d_seg.template as<int32_t>(), w.dslot.as<int>(),
                            st.d_moff.template as<int64_t>(), active, bufs,
                            C.rs.template as<int64_t>(), C.re.template as<int64_t>(),
                            C.col.template as<int32_t>(), reinterpret_cast<double *>(C.val.p), s);
      }
    }
    // a tensor-core wait that gave up leaves the products undefined
    int herr = 0;
    d2h(&herr, w.derr.p, 1, s);
    wait();
    if (herr) throw Error(SIGN_ETIMEOUT, "a bounded wait of the dense tensor-core path gave up");
  }

  // ---------------------------------------------------------------- rounds
  // Re-lays out a stage with its live matrices and the incoming ones.
  template <typename T>
  void rebuild(Stage<T> &st) {
    HostScope hr(KH_REBUILD);
    int nb = int(st.mats.size());
    std::vector<int64_t> eoff(nb + 1, 0);
    if (nb > 0) {
      w.eoff.ensure(sizeof(int64_t) * size_t(nb + 1), s);
      launch_gather_offsets(nb, st.d_moff.template as<int64_t>(), st.X.d_rp(),
                            w.eoff.as<int64_t>(), s);
      d2h(eoff.data(), w.eoff.p, eoff.size(), s);
      wait();
    }
    std::vector<int> mats;
    std::vector<AsmBlock> blocks;
    std::vector<int64_t> bnnz;
    int64_t off = 0;
    for (int i = 0; i < nb; ++i) {
      if (!st.alive[i]) continue;
      int id = st.mats[i];
      blocks.push_back(AsmBlock{st.X.d_rp(), st.X.d_col(), st.X.val.p, st.moff[i],
                                st.moff[i + 1] - st.moff[i], off - st.moff[i], is_f32<T>()});
      bnnz.push_back(eoff[i + 1] - eoff[i]);
      mats.push_back(id);
      off += m[id].h->n;
    }
    for (const auto &p : st.incoming) {
      blocks.push_back(AsmBlock{p->rp, p->col, p->val, p->row0, p->n, off - p->col0, 0});
      bnnz.push_back(p->nnz);
      mats.push_back(p->mat);
      off += p->n;
    }
    Csr<T> nx;
    assemble<T>(blocks, bnnz, nx);
    st.X.swap(nx);
    st.mats = mats;
    st.alive.assign(mats.size(), 1);
    st.ex.assign(1, 0);
    for (int64_t b : bnnz) st.ex.push_back(st.ex.back() + b);
    set_layout(st.moff, st.mats, st.d_moff, st.d_seg);
    st.incoming.clear();  // their buffers are freed in stream order, after the assembly
  }

  template <typename T, typename TN>
  void round(Stage<T> &st, Stage<TN> *next) {
    if (!st.incoming.empty()) rebuild(st);
    int nb = int(st.mats.size());
    int live = 0;
    for (int a : st.alive) live += a;
    if (live == 0) return;
    hm.alloc(nb);
    int64_t N = st.moff.back();
    w.active.ensure(sizeof(int) * size_t(nb), s);
    put(w.active.p, st.alive.data(), st.alive.size());
    const int *d_act = w.active.as<int>();
    const std::vector<int64_t> ex = st.ex;  // entry offsets of the iterate per matrix
    // ---- check: T = X X, r, x, budget (steps a2, a4)
    Rows xr = compact_rows(st.X);
    HostScope hcheck(KH_CHECK);
    DensePlan dp = plan_dense(st);
    product(st, xr, st.X.d_val(), st.X.nnz, xr, st.X.d_val(), st.X.nnz, MODE_SQUARE, st.Tm, d_act,
            &dp);
    std::vector<double> mt(hm.mults, hm.mults + nb);  // sparse multiply-adds of T
    w.sums.ensure(sizeof(double) * size_t(2 * nb), s);
    w.ms.ensure(sizeof(MatScalars) * size_t(nb), s);
    double tol_stage = st.prec == 32 ? o.fp32_until : o.tol;
    {
      ProfScope ps(KC_REDUCE, s);
      launch_seg_reduce(nb, st.d_moff.template as<int64_t>(), w.part.as<double>(), 2,
                        w.sums.as<double>(), s);
      launch_matrix_scalars(nb, st.d_moff.template as<int64_t>(), w.sums.as<double>(), o.c4,
                            tol_stage, o.switch_resid, w.ms.as<MatScalars>(), s);
    }
    if (o.budget_norm) {  // variant: x = ||X||_2 in Eq. (1.18)
      ProfScope ps(KC_REDUCE, s);
      Norm2Work nw{w.n2v.ensure(sizeof(double) * size_t(N), s) ? w.n2v.as<double>() : nullptr,
                   w.n2y.ensure(sizeof(double) * size_t(N), s) ? w.n2y.as<double>() : nullptr,
                   w.n2z.ensure(sizeof(double) * size_t(N), s) ? w.n2z.as<double>() : nullptr,
                   w.n2part.ensure(sizeof(double) * size_t(N), s) ? w.n2part.as<double>() : nullptr,
                   w.n2nrm.ensure(sizeof(double) * size_t(nb), s) ? w.n2nrm.as<double>() : nullptr,
                   w.n2zacc.ensure(sizeof(unsigned long long) * 2 * size_t(N), s)
                       ? w.n2zacc.as<unsigned long long>() : nullptr,
                   w.n2xmax.ensure(sizeof(unsigned long long) * size_t(nb), s)
                       ? w.n2xmax.as<unsigned long long>() : nullptr,
                   w.n2ymax.ensure(sizeof(unsigned long long) * size_t(nb), s)
                       ? w.n2ymax.as<unsigned long long>() : nullptr};
      w.x2.ensure(sizeof(double) * size_t(nb), s);
      launch_norm2_est(nb, st.d_moff.template as<int64_t>(), st.d_seg.template as<int32_t>(), N,
                       xr, st.X.val.p, is_f32<T>(), w.ms.as<MatScalars>(), o.switch_resid, nw,
                       w.x2.as<double>(), s);
      launch_budget_x2(nb, st.d_moff.template as<int64_t>(), w.x2.as<double>(), o.switch_resid,
                       w.ms.as<MatScalars>(), s);
    }
    d2h(hm.ms, w.ms.p, size_t(nb), s);
    d2h(hm.nnz_t, w.nnzc.p, size_t(nb), s);
    std::vector<unsigned long long> dcount(dp.nd);
    if (dp.any()) d2h(dcount.data(), w.dcount.p, size_t(dp.nd), s);
    wait();
    for (int d = 0; d < dp.nd; ++d) {  // the dense path's T: its nonzeros and multiply-adds
      int i = dp.mat[d];
      hm.nnz_t[i] += int64_t(dcount[d]);
      double n = double(st.moff[i + 1] - st.moff[i]);
      mt[i] = n * n * n;
    }
    hcheck.stop();
    std::vector<MatScalars> hms(hm.ms, hm.ms + nb);
    // ---- per-matrix decisions (steps a7, a8); leavers copied out in one launch
    HostScope hdecide(KH_DECIDE);
    int nx = 0;
    int64_t xmax = 0;  // most entries (or rows + 1) of one extracted block
    bool changed = false;
    std::vector<int> movers;
    for (int i = 0; i < nb; ++i) {
      if (!st.alive[i]) continue;
      MatState &ms = m[st.mats[i]];
      double r = hms[i].r;
      trace_put(ms, ex[i + 1] - ex[i], hm.nnz_t[i], r, hms[i].x, st.prec, mt[i]);
      ms.resid = r;
      int decision = 0;  // 0 update, 1 retire, 2 move
      if (st.prec == 64 && r <= o.tol) {
        ms.status = SIGN_OK;
        decision = 1;
      } else if (!std::isfinite(r) || r > o.div_limit) {
        ms.status = SIGN_EDIVERGED;
        decision = 1;
      } else if (st.prec == 32 && r < o.fp32_until) {
        decision = 2;
      } else if (ms.k >= o.max_iter) {
        ms.status = SIGN_ENOTCONV;
        decision = 1;
      }
      if (decision == 0) continue;
      changed = true;
      st.alive[i] = 0;
      if (decision == 2) {
        movers.push_back(i);
        continue;
      }
      int64_t n_i = st.moff[i + 1] - st.moff[i], nnz_i = ex[i + 1] - ex[i];
      Csr<double> *dst = &ms.h->result;
      ms.h->has_result = true;
      retired.push_back(st.mats[i]);
      dst->ensure(n_i, nnz_i, s);
      xmax = std::max(xmax, std::max(nnz_i, n_i + 1));
      hm.xb[nx++] = ExtractBlock{st.X.d_rp(), st.X.d_col(), st.X.val.p, is_f32<T>(), st.moff[i],
                                 n_i, -st.moff[i], dst->d_rp(), dst->d_col(), dst->d_val()};
    }
    if (!movers.empty() && next) {
      // the movers' rows, widened to FP64, one after another in one shared CSR
      // (each with row pointers and columns local to itself)
      int64_t rows = 0, ents = 0;
      for (int i : movers) {
        rows += st.moff[i + 1] - st.moff[i] + 1;
        ents += ex[i + 1] - ex[i];
      }
      auto owner = std::make_shared<Csr<double>>();
      owner->rp.ensure(sizeof(int64_t) * size_t(rows), s);
      owner->col.ensure(sizeof(int32_t) * size_t(ents > 0 ? ents : 1), s);
      owner->val.ensure(sizeof(double) * size_t(ents > 0 ? ents : 1), s);
      int64_t ro = 0, eo = 0;
      for (int i : movers) {
        int64_t n_i = st.moff[i + 1] - st.moff[i], nnz_i = ex[i + 1] - ex[i];
        auto p = std::make_unique<Parked>();
        p->mat = st.mats[i];
        p->owner = owner;
        int64_t *rp = owner->d_rp() + ro;
        int32_t *col = owner->d_col() + eo;
        double *val = owner->d_val() + eo;
        p->rp = rp;
        p->col = col;
        p->val = val;
        p->row0 = 0;
        p->n = n_i;
        p->col0 = 0;
        p->nnz = nnz_i;
        xmax = std::max(xmax, std::max(nnz_i, n_i + 1));
        hm.xb[nx++] = ExtractBlock{st.X.d_rp(), st.X.d_col(), st.X.val.p, is_f32<T>(), st.moff[i],
                                   n_i, -st.moff[i], rp, col, val};
        next->incoming.push_back(std::move(p));
        ro += n_i + 1;
        eo += nnz_i;
      }
    }
    if (nx > 0) {
      w.xblocks.ensure(sizeof(ExtractBlock) * size_t(nx), s);
      h2d(w.xblocks.p, hm.xb, size_t(nx), s);
      ProfScope ps(KC_ASSEMBLE, s);
      launch_extract(nx, w.xblocks.as<ExtractBlock>(), xmax, s);
    }
    live = 0;
    for (int a : st.alive) live += a;
    if (live == 0) {
      wait();  // the extraction reads X and the pinned block list
      return;
    }
    if (changed) put(w.active.p, st.alive.data(), st.alive.size());
    hdecide.stop();
    // ---- update: Xbar = 1.5 X - 0.5 X T (step a3), or NMF's (X + X^-1) / 2
    HostScope hupdate(KH_UPDATE);
    int64_t nnz_t_all = 0;
    for (int i = 0; i < nb; ++i) nnz_t_all += hm.nnz_t[i];
    std::vector<double> mb(nb, 0.0);
    bool nmf = false;
    if constexpr (sizeof(T) == 8) nmf = o.method == SIGN_METHOD_NMF;
    if (nmf) {
      if constexpr (sizeof(T) == 8) {
        if (!nmf_update(st, d_act)) return;  // every updating iterate was singular
      }
    } else if (o.filter_t && o.filter != SIGN_FILTER_NONE) {
      // variant: T filtered with the same budget and filter before the update
      select_threshold(st, st.Tm, d_act);
      std::vector<int64_t> tex;
      filter_rows(st, st.Tm, st.Th, d_act, tex, nullptr);
      for (int i = 0; i < nb; ++i)
        if (st.alive[i]) trace_that(m[st.mats[i]], tex[i + 1] - tex[i]);
      product(st, xr, st.X.d_val(), st.X.nnz, compact_rows(st.Th), st.Th.d_val(), st.Th.nnz,
              MODE_UPDATE, st.Xb, d_act, &dp, false);
    } else {
      product(st, xr, st.X.d_val(), st.X.nnz, st.Tm.rows(), st.Tm.d_val(), nnz_t_all,
              MODE_UPDATE, st.Xb, d_act, &dp);
    }
    if (!nmf) {
      mb.assign(hm.mults, hm.mults + nb);
      for (int d = 0; d < dp.nd; ++d) {
        double n = double(st.moff[dp.mat[d] + 1] - st.moff[dp.mat[d]]);
        mb[dp.mat[d]] = n * n * n;
      }
    }
    // per-matrix nnz(Xbar) straight into the device scalars (BOUND needs it)
    launch_store_nnz_bar(nb, w.nnzc.as<int64_t>(), w.ms.as<MatScalars>(), s);
    // the iterate is not read again this round: a large one's memory can take
    // the filtered update (reuse is ordered after the update on this stream)
    if (st.X.col.cap + st.X.val.cap > BIG_BUFFER) {
      st.X.col.release();
      st.X.val.release();
    }
    hupdate.stop();
    HostScope hfilter(KH_FILTER);
    if (o.filter == SIGN_FILTER_NONE) {
      // keep every entry: compact the slotted rows as they are
      hms_none(st, hms);
    } else {
      // ---- threshold (step a5); nnz(Xbar) is in the scalars for BOUND
      select_threshold(st, st.Xb, d_act);
      filter(st, d_act, hms);
    }
    if (st.Xb.col.cap + st.Xb.val.cap > BIG_BUFFER) {  // large update slots: memory for others
      st.Xb.col.release();
      st.Xb.val.release();
    }
    for (int i = 0; i < nb; ++i) {
      if (!st.alive[i]) continue;
      MatState &ms = m[st.mats[i]];
      trace_filter(ms, hms[i].beta, o.filter == SIGN_FILTER_NONE ? 0.0 : hms[i].tau,
                   o.filter == SIGN_FILTER_NONE ? 0.0 : hms[i].fnorm, hms[i].nnz_bar, mb[i]);
      ms.k++;
    }
    st.X.swap(st.Xh);
  }

  // Threshold (step a5) of each active matrix over the values of `in`, into
  // the device scalars: EXACT by the radix select, BOUND by b/sqrt(nnz) with
  // nnz the last product's per-matrix count (launch_seg_count). EXACT also
  // leaves the filter's per-row counts and dropped squares in w.cnt and
  // w.dropped (filter_rows reads them instead of counting again).
  // NMF (Alg. 3.1.1) in place of the Newton-Schulz update, FP64 stage: for
  // every updating matrix the dense inverse of its iterate, Xbar = (X +
  // X^-1) / 2 into full rows of slots of st.Xb and the budget of Eq. (1.13).
  // A matrix whose iterate is singular stops with SIGN_EDIVERGED, its
  // iterate as the result. Returns false if no matrix is left to filter.
  bool nmf_update(Stage<double> &st, const int *d_act) {
    const int nb = int(st.mats.size());
    const int64_t N = st.moff.back();
    int64_t slots = 0, nmax = 0;
    for (int i = 0; i < nb; ++i)
      if (st.alive[i]) {
        const int64_t n = st.moff[i + 1] - st.moff[i];
        slots += n * n;
        nmax = std::max(nmax, n);
      }
    Slotted<double> &C = st.Xb;
    C.n = N;
    C.slots = slots;
    C.rs.ensure(sizeof(int64_t) * size_t(N + 1), s);
    C.re.ensure(sizeof(int64_t) * size_t(N > 0 ? N : 1), s);
    C.col.ensure(sizeof(int32_t) * size_t(slots > 0 ? slots : 1), s);
    C.val.ensure(sizeof(double) * size_t(slots > 0 ? slots : 1), s);
    SGN_CUDA(cudaMemsetAsync(C.rs.p, 0, sizeof(int64_t) * size_t(N + 1), s));
    SGN_CUDA(cudaMemsetAsync(C.re.p, 0, sizeof(int64_t) * size_t(N > 0 ? N : 1), s));
    const size_t blk = size_t(nmax) * size_t(nmax);
    double *dx = static_cast<double *>(w.dmem.ensure(sizeof(double) * (3 * blk + size_t(nmax)), s));
    double *lu = dx + blk, *inv = lu + blk, *part = inv + blk;
    w.nmf_int.ensure(sizeof(int) * size_t(nmax + 2 + nb), s);
    w.nmf_dbl.ensure(sizeof(double) * size_t(nb), s);
    int *perm = w.nmf_int.as<int>(), *pivot = perm + nmax, *sing = pivot + 2;
    double *xinv = w.nmf_dbl.as<double>();
    SGN_CUDA(cudaMemsetAsync(sing, 0, sizeof(int) * size_t(nb), s));
    int64_t slot0 = 0;
    for (int i = 0; i < nb; ++i) {
      if (!st.alive[i]) continue;
      const int64_t row0 = st.moff[i], n = st.moff[i + 1] - row0;
      const int ni = int(n);
      ProfScope ps(KC_DENSE64, s, 2.0 * double(n) * double(n) * double(n), 0.0);
      SGN_CUDA(cudaMemsetAsync(dx, 0, sizeof(double) * size_t(n) * size_t(n), s));
      launch_nmf_densify(ni, ni, st.X.d_rp(), st.X.d_col(), st.X.d_val(), row0, dx, s);
      SGN_CUDA(cudaMemcpyAsync(lu, dx, sizeof(double) * size_t(n) * size_t(n),
                               cudaMemcpyDeviceToDevice, s));
      launch_dense_inverse(ni, ni, lu, perm, pivot, sing + i, inv, s);
      launch_inv_norm(ni, ni, inv, part, xinv + i, s);
      launch_nmf_combine(ni, ni, dx, inv, row0, slot0, C.rs.as<int64_t>(), C.re.as<int64_t>(),
                         C.col.as<int32_t>(), C.val.as<double>(), s);
      launch_nmf_budget(i, n, xinv + i, o.c4, o.tol, o.switch_resid, w.ms.as<MatScalars>(), s);
      slot0 += n * n;
    }
    std::vector<int> hsing(nb, 0);
    d2h(hsing.data(), sing, size_t(nb), s);
    wait();
    // singular iterates stop here, their iterate as the result
    int nx = 0;
    int64_t xmax = 0;
    for (int i = 0; i < nb; ++i) {
      if (!st.alive[i] || !hsing[i]) continue;
      MatState &ms = m[st.mats[i]];
      ms.status = SIGN_EDIVERGED;
      st.alive[i] = 0;
      const int64_t n_i = st.moff[i + 1] - st.moff[i], nnz_i = st.ex[i + 1] - st.ex[i];
      Csr<double> *dst = &ms.h->result;
      ms.h->has_result = true;
      retired.push_back(st.mats[i]);
      dst->ensure(n_i, nnz_i, s);
      xmax = std::max(xmax, std::max(nnz_i, n_i + 1));
      hm.xb[nx++] = ExtractBlock{st.X.d_rp(), st.X.d_col(), st.X.val.p, 0, st.moff[i], n_i,
                                 -st.moff[i], dst->d_rp(), dst->d_col(), dst->d_val()};
    }
    if (nx > 0) {
      w.xblocks.ensure(sizeof(ExtractBlock) * size_t(nx), s);
      h2d(w.xblocks.p, hm.xb, size_t(nx), s);
      launch_extract(nx, w.xblocks.as<ExtractBlock>(), xmax, s);
      put(w.active.p, st.alive.data(), st.alive.size());
    }
    launch_seg_count(nb, st.d_moff.template as<int64_t>(), C.rs.as<int64_t>(), C.re.as<int64_t>(),
                     w.nnzc.as<int64_t>(), s);
    launch_store_nnz_bar(nb, w.nnzc.as<int64_t>(), w.ms.as<MatScalars>(), s);
    int live = 0;
    for (int a : st.alive) live += a;
    if (live == 0) wait();  // the extraction reads X and the pinned block list
    (void)d_act;
    return live > 0;
  }

  // Above 2^28 values the candidate room is a sixteenth of them (at least
  // 2^28); filter_rows selects again with full room if the crossing bucket
  // held more.
  template <typename T>
  void select_threshold(Stage<T> &st, Slotted<T> &in, const int *d_act, bool full_room = false) {
    int64_t N = st.moff.back();
    int nb = int(st.mats.size());
    if (o.filter == SIGN_FILTER_EXACT) {
      const int64_t big = int64_t(1) << 28;
      w.sel_cap = full_room || in.slots <= big ? in.slots : std::max(big, in.slots / 16);
      w.sel.ensure(select_scratch_bytes(nb, w.sel_cap), s);
      w.dropped.ensure(sizeof(double) * size_t(N > 0 ? N : 1), s);
      w.cnt.ensure(sizeof(int64_t) * size_t(N > 0 ? N : 1), s);
      SelRows R{N, st.d_seg.template as<int32_t>(), in.rs.template as<int64_t>(),
                in.re.template as<int64_t>(), 0};
      launch_select_exact(nb, R, w.sel_cap, d_act, in.val.p, is_f32<T>(), w.ms.as<MatScalars>(),
                          w.sel.p, w.cnt.as<int64_t>(), w.dropped.as<double>(), s);
    } else {
      ProfScope psel(KC_SELECT, s);
      launch_store_nnz_bar(nb, w.nnzc.as<int64_t>(), w.ms.as<MatScalars>(), s);
      launch_select_bound(nb, d_act, w.ms.as<MatScalars>(), s);
    }
  }

  // Filter + compaction (step a6) of the slotted rows `in` into the compact
  // `out`: the entries with |x| >= tau and x != 0. ex receives the entry
  // offsets of the matrices; dsum (nullable) the dropped sums of squares.
  template <typename T>
  void filter_rows(Stage<T> &st, Slotted<T> &in, Csr<T> &out, const int *d_act,
                   std::vector<int64_t> &ex, std::vector<double> *dsum) {
    int64_t N = st.moff.back();
    int nb = int(st.mats.size());
    w.dropped.ensure(sizeof(double) * size_t(N > 0 ? N : 1), s);
    w.cnt.ensure(sizeof(int64_t) * size_t(N > 0 ? N : 1), s);
    out.rp.ensure(sizeof(int64_t) * size_t(N + 1), s);
    w.eoff.ensure(sizeof(int64_t) * size_t(nb + 1), s);
    const bool exact = o.filter == SIGN_FILTER_EXACT;
    for (;;) {
      {
        // EXACT: the select counted already (all but the crossing buckets' squares)
        ProfScope pf(KC_FILTER, s, 0.0,
                     (exact ? 0.0 : double(in.slots) * sizeof(T)) + 24.0 * double(N));
        if (!exact)
          launch_filter_count(N, st.d_seg.template as<int32_t>(), d_act,
                              in.rs.template as<int64_t>(), in.re.template as<int64_t>(),
                              in.val.p, is_f32<T>(), w.ms.as<MatScalars>(), w.cnt.as<int64_t>(),
                              w.dropped.as<double>(), s);
        launch_scan(N, w.cnt.as<int64_t>(), out.d_rp(), w.scan_tmp.as<int64_t>(), s);
        launch_seg_reduce(nb, st.d_moff.template as<int64_t>(), w.dropped.as<double>(), 1,
                          w.sums.as<double>(), s);
        if (exact)
          launch_select_drop_fix(nb, d_act, w.sel.p, w.ms.as<MatScalars>(), w.sums.as<double>(),
                                 s);
        launch_gather_offsets(nb, st.d_moff.template as<int64_t>(), out.d_rp(),
                              w.eoff.as<int64_t>(), s);
      }
      d2h(hm.ex, w.eoff.p, size_t(nb + 1), s);
      d2h(hm.tot, out.d_rp() + N, 1, s);
      d2h(hm.ms, w.ms.p, size_t(nb), s);
      d2h(hm.dsum, w.sums.p, size_t(nb), s);
      const bool capped = exact && w.sel_cap < in.slots;
      if (capped) d2h(reinterpret_cast<unsigned long long *>(hm.tot + 3),
                      select_cand_count(w.sel.p, nb), 1, s);
      wait();
      if (!capped || uint64_t(hm.tot[3]) <= uint64_t(w.sel_cap)) break;
      select_threshold(st, in, d_act, true);  // the crossing bucket outgrew the room
    }
    int64_t nnz = hm.tot[0];
    out.n = N;
    out.nnz = nnz;
    out.col.ensure(sizeof(int32_t) * size_t(nnz > 0 ? nnz : 1), s);
    out.val.ensure(sizeof(T) * size_t(nnz > 0 ? nnz : 1), s);
    {
      ProfScope pw(KC_FILTER, s, 0.0,
                   double(in.slots + nnz) * (sizeof(T) + 4.0) + 24.0 * double(N));
      launch_filter_write(N, st.d_seg.template as<int32_t>(), d_act, in.rs.template as<int64_t>(),
                          in.re.template as<int64_t>(), in.col.template as<int32_t>(), in.val.p,
                          is_f32<T>(), w.ms.as<MatScalars>(), out.d_rp(), out.d_col(), out.val.p,
                          s);
    }
    ex.assign(hm.ex, hm.ex + nb + 1);
    if (dsum) dsum->assign(hm.dsum, hm.dsum + nb);
  }

  // Filter + compaction (step a6): Xh = entries of Xb with |x| >= tau, x != 0.
  template <typename T>
  void filter(Stage<T> &st, const int *d_act, std::vector<MatScalars> &hms) {
    int nb = int(st.mats.size());
    std::vector<int64_t> ex;
    std::vector<double> dsum;
    filter_rows(st, st.Xb, st.Xh, d_act, ex, &dsum);
    for (int i = 0; i < nb; ++i) {
      hms[i].tau = hm.ms[i].tau;
      hms[i].nnz_bar = hm.ms[i].nnz_bar;
      hms[i].beta = hm.ms[i].beta;  // NMF sets its own budget after the check
      hms[i].fnorm = std::sqrt(dsum[i]);
    }
    st.ex = ex;
  }

  // No filter: the update is compacted with every entry kept (exact zeros too).
  template <typename T>
  void hms_none(Stage<T> &st, std::vector<MatScalars> &hms) {
    int64_t N = st.moff.back();
    w.cnt.ensure(sizeof(int64_t) * size_t(N > 0 ? N : 1), s);
    ProfScope pf(KC_FILTER, s, 0.0, double(st.Xb.slots) * (2.0 * sizeof(T) + 8.0));
    launch_row_lengths(N, st.Xb.rs.template as<int64_t>(), st.Xb.re.template as<int64_t>(),
                       w.cnt.as<int64_t>(), s);
    st.Xh.rp.ensure(sizeof(int64_t) * size_t(N + 1), s);
    launch_scan(N, w.cnt.as<int64_t>(), st.Xh.d_rp(), w.scan_tmp.as<int64_t>(), s);
    int nbm = int(st.mats.size());
    w.eoff.ensure(sizeof(int64_t) * size_t(nbm + 1), s);
    launch_gather_offsets(nbm, st.d_moff.template as<int64_t>(), st.Xh.d_rp(), w.eoff.as<int64_t>(), s);
    d2h(hm.ex, w.eoff.p, size_t(nbm + 1), s);
    d2h(hm.tot, st.Xh.d_rp() + N, 1, s);
    d2h(hm.ms, w.ms.p, size_t(nbm), s);
    wait();
    for (int i = 0; i < nbm; ++i) {
      hms[i].nnz_bar = hm.ms[i].nnz_bar;
      hms[i].beta = hm.ms[i].beta;  // NMF sets its own budget after the check
    }
    st.ex.assign(hm.ex, hm.ex + nbm + 1);
    int64_t nnz = hm.tot[0];
    st.Xh.n = N;
    st.Xh.nnz = nnz;
    st.Xh.col.ensure(sizeof(int32_t) * size_t(nnz > 0 ? nnz : 1), s);
    st.Xh.val.ensure(sizeof(T) * size_t(nnz > 0 ? nnz : 1), s);
    launch_compact_rows(N, st.Xb.rs.template as<int64_t>(), st.Xb.re.template as<int64_t>(),
                        st.Xb.col.template as<int32_t>(), st.Xb.val.p, sizeof(T), st.Xh.d_rp(),
                        st.Xh.d_col(), st.Xh.val.p, s);
  }

  // ---------------------------------------------------------------- admission
  // Takes matrices into the solve (step a1). Their inputs, assembled into one
  // block-diagonal FP64 CSR, are scaled by their 1-norms and parked for the
  // entry stage (FP32 in the mixed mode), which they join at its next round.
  // A matrix without a finite nonzero 1-norm fails the call when strict, else
  // it stops at once with SIGN_EINVAL. Returns the ids given to the matrices.
  std::vector<int> admit(const std::vector<sign_t> &hs, const std::vector<sign_info *> &infos,
                         bool strict) {
    const int count = int(hs.size());
    std::vector<int> ids(count);
    for (int i = 0; i < count; ++i) {
      int id;
      if (!free_ids.empty()) {
        id = free_ids.back();
        free_ids.pop_back();
      } else {
        id = int(m.size());
        m.emplace_back();
      }
      m[id] = MatState{};
      m[id].h = hs[i];
      m[id].info = infos.empty() ? nullptr : infos[i];
      hs[i]->has_result = false;
      ids[i] = id;
    }
    if (o.method == SIGN_METHOD_NMF)
      for (int i = 0; i < count; ++i)
        if (hs[i]->n > NMF_MAX_N)
          throw Error(SIGN_EINVAL, "NMF: matrix " + std::to_string(i) + " is larger than " +
                                       std::to_string(NMF_MAX_N) + " (dense inverse)");
    HostScope hsetup(KH_SETUP);
    std::vector<AsmBlock> blocks;
    std::vector<int64_t> bnnz, moff;
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
      blocks.push_back(AsmBlock{hs[i]->a.d_rp(), hs[i]->a.d_col(), hs[i]->a.val.p, 0, hs[i]->n, off, 0});
      bnnz.push_back(hs[i]->nnz);
      off += hs[i]->n;
    }
    auto owner = std::make_shared<Csr<double>>();
    assemble<double>(blocks, bnnz, *owner);
    DevBuf d_moff, d_seg;
    set_layout(moff, ids, d_moff, d_seg);
    const int64_t N = off;
    std::vector<char> ok(count, 1);
    if (o.scale_1norm && o.method != SIGN_METHOD_NMF) {  // NMF starts from X_1 = A
      w.norm_work.ensure(sizeof(unsigned long long) * size_t(2 * N + 4 * count), s);
      w.norm.ensure(sizeof(double) * size_t(count), s);
      std::vector<double> nrm(count);
      {
        ProfScope ps(KC_NORM, s);
        launch_onenorm(count, d_moff.as<int64_t>(), d_seg.as<int32_t>(), N, owner->d_rp(),
                       owner->d_col(), owner->d_val(), w.norm_work.as<unsigned long long>(),
                       w.norm.as<double>(), s);
      }
      d2h(nrm.data(), w.norm.p, size_t(count), s);
      wait();
      for (int i = 0; i < count; ++i)
        if (!(nrm[i] > 0.0) || !std::isfinite(nrm[i])) {
          if (strict)
            throw Error(SIGN_EINVAL, "matrix " + std::to_string(i) + " has no finite nonzero 1-norm");
          ok[i] = 0;
          m[ids[i]].status = SIGN_EINVAL;
          retired.push_back(ids[i]);
        }
      launch_scale(N, d_seg.as<int32_t>(), owner->d_rp(), owner->d_val(), w.norm.as<double>(), s);
    }
    for (int i = 0; i < count; ++i) {
      if (!ok[i]) continue;
      auto p = std::make_unique<Parked>();
      p->mat = ids[i];
      p->owner = owner;
      p->rp = owner->d_rp();
      p->col = owner->d_col();
      p->val = owner->d_val();
      p->row0 = moff[i];
      p->n = hs[i]->n;
      p->col0 = moff[i];
      p->nnz = hs[i]->nnz;
      if (o.prec == SIGN_PREC_MIXED)
        s32.incoming.push_back(std::move(p));
      else
        s64.incoming.push_back(std::move(p));
    }
    return ids;
  }

  // One round of each stage; the FP32 stage's movers enter FP64 in the same step.
  // A stage left without matrices hands large buffers back (to this thread's
  // block cache and the pool), so that the other stage can use the memory;
  // small ones are kept for the next solve.
  void step() {
    round<float, double>(s32, &s64);
    if (s32.incoming.empty() && !has_live(s32) && stage_bytes(s32) > BIG_BUFFER) release_stage(s32);
    round<double, double>(s64, nullptr);
    if (s64.incoming.empty() && !has_live(s64) && stage_bytes(s64) > BIG_BUFFER) release_stage(s64);
  }

  template <typename T>
  static size_t stage_bytes(const Stage<T> &st) {
    size_t b = 0;
    for (const Csr<T> *c : {&st.X, &st.Xh, &st.Th}) b += c->rp.cap + c->col.cap + c->val.cap;
    for (const Slotted<T> *c : {&st.Tm, &st.Xb}) b += c->rs.cap + c->re.cap + c->col.cap + c->val.cap;
    return b;
  }

  template <typename T>
  static bool has_live(const Stage<T> &st) {
    for (int a : st.alive)
      if (a) return true;
    return false;
  }

  // The stage then holds no matrix at all (a later admission rebuilds it from
  // its incoming matrices alone, reading none of the released buffers).
  template <typename T>
  void release_stage(Stage<T> &st) {
    st.mats.clear();
    st.alive.clear();
    st.moff.assign(1, 0);
    st.ex.assign(1, 0);
    for (Csr<T> *c : {&st.X, &st.Xh, &st.Th}) {
      c->rp.release();
      c->col.release();
      c->val.release();
      c->n = c->nnz = 0;
    }
    for (Slotted<T> *c : {&st.Tm, &st.Xb}) {
      c->rs.release();
      c->re.release();
      c->col.release();
      c->val.release();
      c->n = c->slots = 0;
    }
  }

  bool busy() const {
    if (!s32.incoming.empty() || !s64.incoming.empty()) return true;
    for (int a : s32.alive)
      if (a) return true;
    for (int a : s64.alive)
      if (a) return true;
    return false;
  }

  // Ids of the matrices that stopped since the last call. Their MatState stays
  // readable until the next admit, which may reuse the ids.
  std::vector<int> collect() {
    std::vector<int> r;
    r.swap(retired);
    free_ids.insert(free_ids.end(), r.begin(), r.end());
    return r;
  }

  // ---------------------------------------------------------------- solve
  void run(sign_t *hs, int count, sign_info *infos) {
    hm.alloc(count);
    std::vector<sign_t> v(hs, hs + count);
    std::vector<sign_info *> in;
    if (infos)
      for (int i = 0; i < count; ++i) in.push_back(&infos[i]);
    std::vector<int> ids = admit(v, in, true);
    for (int guard = 0; guard < 4 * o.max_iter + 16 && busy(); ++guard) step();
    wait();
    for (int i = 0; i < count; ++i) {
      MatState &ms = m[ids[i]];
      if (ms.status < 0) throw Error(SIGN_ESTATE, "solve loop ended with a running matrix");
      if (ms.info) {
        ms.info->iters = ms.k;
        ms.info->status = ms.status;
        ms.info->resid = ms.resid;
        ms.info->nnz_final = hs[i]->result.nnz;
        ms.info->count = ms.trace_count;
      }
    }
  }
};

}  // namespace
