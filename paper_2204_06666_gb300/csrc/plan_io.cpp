// Plan files: the host arrays of a plan (partition, permutation, slab and ER encoding), written once and
// loaded later without partitioning and encoding again -- the preprocessing whose cost the paper weighs
// against the many SpMVs of a solver (Sec. 6).  A loaded plan is uploaded like a freshly built one.
//
// Layout (native little-endian, the machine that writes is the machine family that reads):
//   FileHeader, then kArrays arrays back to back in the order of for_each_array, each len[i] elements.
//   checksum = FNV-1a over the payload taken as 64-bit words (a short last word is zero-padded).
// A file is untrusted input: before anything is uploaded, every structural invariant the kernels rely on
// (a permutation, monotone pointers, slice widths, local column offsets inside their partition, global
// columns inside [0, n)) is checked, so a corrupt file gives EHYB_ERR_IO and never a device fault.
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "plan_internal.h"

namespace ehyb {
namespace {

constexpr char kMagic[8] = {'E', 'H', 'Y', 'B', 'P', 'L', 'A', 'N'};
constexpr uint32_t kVersion = 1;
constexpr int kArrays = 18;

struct FileHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int64_t n, nnz, er_nnz, ell_nnz;
  int32_t nparts, nslices, tpr, slice_rows, er_layout, max_part_rows, tuner_path, ell_width_cap;
  int64_t len[kArrays];
  uint64_t checksum;
};

// visit the arrays of a host plan in file order: f(vector&)
template <typename H, typename F>
void for_each_array(H& P, F&& f) {
  f(P.new_to_old);
  f(P.part_ptr);
  f(P.slice_ptr);
  f(P.slice_pos);
  f(P.slice_order);
  f(P.ell_col);
  f(P.ell_val);
  f(P.row_ell_count);
  f(P.er_part_ptr);
  f(P.er_row);
  f(P.er_ptr);
  f(P.er_col);
  f(P.er_val);
  f(P.er_slice_pos);
  f(P.er_scol);
  f(P.er_scol_old);
  f(P.er_sval);
  f(P.row_er_count);
}

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  uint8_t tail[8];
  int nt = 0;
  void word(uint64_t w) { h = (h ^ w) * 1099511628211ull; }
  void add(const void* p, size_t bytes) {
    const uint8_t* b = (const uint8_t*)p;
    while (bytes && nt) {  // complete a pending word
      tail[nt++] = *b++;
      --bytes;
      if (nt == 8) {
        uint64_t w;
        std::memcpy(&w, tail, 8);
        word(w);
        nt = 0;
      }
    }
    for (; bytes >= 8; bytes -= 8, b += 8) {
      uint64_t w;
      std::memcpy(&w, b, 8);
      word(w);
    }
    while (bytes--) tail[nt++] = *b++;
  }
  uint64_t done() {
    if (nt) {
      std::memset(tail + nt, 0, (size_t)(8 - nt));
      uint64_t w;
      std::memcpy(&w, tail, 8);
      word(w);
      nt = 0;
    }
    return h;
  }
};

struct File {
  FILE* f = nullptr;
  explicit File(FILE* p) : f(p) {}
  ~File() {
    if (f) std::fclose(f);
  }
};

bool monotone_from_zero(const std::vector<int32_t>& v) {
  if (v.empty() || v[0] != 0) return false;
  for (size_t i = 1; i < v.size(); ++i)
    if (v[i] < v[i - 1]) return false;
  return true;
}
bool monotone_from_zero(const std::vector<int64_t>& v) {
  if (v.empty() || v[0] != 0) return false;
  for (size_t i = 1; i < v.size(); ++i)
    if (v[i] < v[i - 1]) return false;
  return true;
}

// every invariant the kernels index by
bool valid(const HostPlan& P, const FileHeader& h) {
  const int64_t n = P.n;
  if (n < 0 || n >= (int64_t)INT32_MAX - 1 || P.nparts < 0 || P.nslices < 0) return false;
  if (P.tpr < 1 || P.tpr > 32 || (P.tpr & (P.tpr - 1))) return false;
  if (P.er_layout != 0 && P.er_layout != 1) return false;
  if ((int64_t)P.new_to_old.size() != n || (int64_t)P.row_ell_count.size() != n ||
      (int64_t)P.row_er_count.size() != n)
    return false;
  {
    std::vector<uint8_t> seen((size_t)n, 0);
    for (int32_t v : P.new_to_old) {
      if (v < 0 || v >= n || seen[(size_t)v]) return false;
      seen[(size_t)v] = 1;
    }
  }
  if ((int64_t)P.part_ptr.size() != (int64_t)P.nparts + 1 || !monotone_from_zero(P.part_ptr) ||
      P.part_ptr.back() != n)
    return false;
  int32_t maxr = 0;
  for (int32_t p = 0; p < P.nparts; ++p) maxr = std::max(maxr, P.part_ptr[(size_t)p + 1] - P.part_ptr[(size_t)p]);
  if (maxr != P.max_part_rows || maxr > 65536) return false;
  const int rps = 32 / P.tpr;
  if ((int64_t)P.slice_ptr.size() != (int64_t)P.nparts + 1 || !monotone_from_zero(P.slice_ptr) ||
      P.slice_ptr.back() != P.nslices)
    return false;
  for (int32_t p = 0; p < P.nparts; ++p) {
    const int32_t rows = P.part_ptr[(size_t)p + 1] - P.part_ptr[(size_t)p];
    if (P.slice_ptr[(size_t)p + 1] - P.slice_ptr[(size_t)p] != (rows + rps - 1) / rps) return false;
  }
  if ((int64_t)P.slice_pos.size() != (int64_t)P.nslices + 1 || !monotone_from_zero(P.slice_pos)) return false;
  if ((int64_t)P.ell_col.size() != P.slice_pos.back() || P.ell_val.size() != P.ell_col.size()) return false;
  if ((int64_t)P.slice_order.size() != P.nslices) return false;
  for (int32_t p = 0; p < P.nparts; ++p) {
    const int32_t s0 = P.slice_ptr[(size_t)p], s1 = P.slice_ptr[(size_t)p + 1];
    const int32_t rows = P.part_ptr[(size_t)p + 1] - P.part_ptr[(size_t)p];
    std::vector<uint8_t> seen((size_t)(s1 - s0), 0);
    for (int32_t i = s0; i < s1; ++i) {
      const int32_t s = P.slice_order[(size_t)i];
      if (s < s0 || s >= s1 || seen[(size_t)(s - s0)]) return false;
      seen[(size_t)(s - s0)] = 1;
    }
    for (int32_t s = s0; s < s1; ++s) {
      const int64_t a = P.slice_pos[(size_t)s], b = P.slice_pos[(size_t)s + 1];
      if ((b - a) % 32) return false;
      for (int64_t k = a; k < b; ++k)
        if ((int32_t)P.ell_col[(size_t)k] >= rows) return false;
    }
  }
  if (P.er_layout == 0) {
    if ((int64_t)P.er_slice_pos.size() != (int64_t)P.nslices + 1 || !monotone_from_zero(P.er_slice_pos)) return false;
    const size_t es = (size_t)P.er_slice_pos.back();
    if (P.er_scol.size() != es || P.er_scol_old.size() != es || P.er_sval.size() != es) return false;
    for (int32_t s = 0; s < P.nslices; ++s)
      if ((P.er_slice_pos[(size_t)s + 1] - P.er_slice_pos[(size_t)s]) % 32) return false;
    for (size_t k = 0; k < es; ++k) {
      const int32_t c = P.er_scol[k];
      if (c < 0 || c >= n || P.er_scol_old[k] != P.new_to_old[(size_t)c]) return false;
    }
    if (!P.er_row.empty() || !P.er_col.empty() || !P.er_val.empty()) return false;
    if ((int64_t)P.er_part_ptr.size() != (int64_t)P.nparts + 1 || P.er_ptr.size() != 1 || P.er_ptr[0] != 0) return false;
    for (int32_t v : P.er_part_ptr)
      if (v != 0) return false;
  } else {
    if ((int64_t)P.er_part_ptr.size() != (int64_t)P.nparts + 1 || !monotone_from_zero(P.er_part_ptr) ||
        (size_t)P.er_part_ptr.back() != P.er_row.size())
      return false;
    for (int32_t p = 0; p < P.nparts; ++p)
      for (int32_t e = P.er_part_ptr[(size_t)p]; e < P.er_part_ptr[(size_t)p + 1]; ++e) {
        const int32_t r = P.er_row[(size_t)e];
        if (r < P.part_ptr[(size_t)p] || r >= P.part_ptr[(size_t)p + 1]) return false;
      }
    if (P.er_ptr.size() != P.er_row.size() + 1 || !monotone_from_zero(P.er_ptr)) return false;
    if ((size_t)P.er_ptr.back() != P.er_col.size() || P.er_val.size() != P.er_col.size()) return false;
    for (int32_t c : P.er_col)
      if (c < 0 || c >= n) return false;
    if (!P.er_scol.empty() || !P.er_sval.empty()) return false;
    if (P.er_slice_pos.size() != (size_t)P.nslices + 1) return false;
  }
  int64_t ell_nnz = 0, er_nnz = 0;
  for (int64_t r = 0; r < n; ++r) {
    if (P.row_ell_count[(size_t)r] < 0 || P.row_er_count[(size_t)r] < 0) return false;
    ell_nnz += P.row_ell_count[(size_t)r];
    er_nnz += P.row_er_count[(size_t)r];
  }
  if (ell_nnz != h.ell_nnz || er_nnz != h.er_nnz || ell_nnz + er_nnz != h.nnz) return false;
  return true;
}

// the bulky arrays of a plan that dropped them after upload, read back from the device
ehyb_status_t fetch_host_arrays(ehyb_plan_t p, HostPlan& H) {
  if (p->host_kept) return EHYB_OK;
  const DevPlan& D = p->dev;
  const bool sl = p->er_layout == 0;
  try {
    H.ell_col.resize((size_t)p->ell_stored);
    H.ell_val.resize((size_t)p->ell_stored);
    H.er_col.resize(sl ? 0 : (size_t)p->er_nnz);
    H.er_val.resize(sl ? 0 : (size_t)p->er_nnz);
    H.er_scol.resize(sl ? (size_t)p->er_stored : 0);
    H.er_scol_old.resize(sl ? (size_t)p->er_stored : 0);
    H.er_sval.resize(sl ? (size_t)p->er_stored : 0);
  } catch (const std::bad_alloc&) {
    return EHYB_ERR_OOM;
  }
  auto get = [](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) : cudaSuccess;
  };
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = get(H.ell_col.data(), D.ell_col, H.ell_col.size() * 2);
  if (e == cudaSuccess) e = get(H.ell_val.data(), D.ell_val, H.ell_val.size() * 8);
  if (e == cudaSuccess) e = get(H.er_col.data(), D.er_col, H.er_col.size() * 4);
  if (e == cudaSuccess) e = get(H.er_val.data(), D.er_val, H.er_val.size() * 8);
  if (e == cudaSuccess) e = get(H.er_scol.data(), D.er_scol, H.er_scol.size() * 4);
  if (e == cudaSuccess) e = get(H.er_scol_old.data(), D.er_scol_old, H.er_scol_old.size() * 4);
  if (e == cudaSuccess) e = get(H.er_sval.data(), D.er_sval, H.er_sval.size() * 8);
  return e == cudaSuccess ? EHYB_OK : cuda_error_status(e, "plan save: device read");
}

}  // namespace
}  // namespace ehyb

using namespace ehyb;

extern "C" ehyb_status_t ehyb_plan_save(ehyb_plan_t p, const char* path) {
  if (!p || !path) return EHYB_ERR_INVALID_ARG;
  if (p->er_layout == 2) return EHYB_ERR_UNSUPPORTED;  // the file holds no halo
  // a copy of the metadata plus the bulky arrays (from the host copy when kept, else from the device)
  HostPlan tmp;
  const HostPlan* src = &p->host;
  if (!p->host_kept) {
    const HostPlan& H = p->host;
    tmp.new_to_old = H.new_to_old;
    tmp.part_ptr = H.part_ptr;
    tmp.slice_ptr = H.slice_ptr;
    tmp.slice_pos = H.slice_pos;
    tmp.slice_order = H.slice_order;
    tmp.row_ell_count = H.row_ell_count;
    tmp.er_part_ptr = H.er_part_ptr;
    tmp.er_row = H.er_row;
    tmp.er_ptr = H.er_ptr;
    tmp.er_slice_pos = H.er_slice_pos;
    tmp.row_er_count = H.row_er_count;
    ehyb_status_t st = fetch_host_arrays(p, tmp);
    if (st != EHYB_OK) return st;
    src = &tmp;
  }
  const HostPlan& H = p->host;
  FileHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = (uint32_t)sizeof(FileHeader);
  h.n = H.n;
  h.nnz = H.ell_nnz + H.er_nnz;
  h.er_nnz = H.er_nnz;
  h.ell_nnz = H.ell_nnz;
  h.nparts = H.nparts;
  h.nslices = H.nslices;
  h.tpr = H.tpr;
  h.slice_rows = H.slice_rows;
  h.er_layout = H.er_layout;
  h.max_part_rows = H.max_part_rows;
  h.tuner_path = p->tuner_path;
  h.ell_width_cap = p->ell_width_cap;
  int i = 0;
  Fnv fnv;
  for_each_array(*src, [&](const auto& v) {
    h.len[i++] = (int64_t)v.size();
    fnv.add(v.data(), v.size() * sizeof(v[0]));
  });
  h.checksum = fnv.done();
  File f(std::fopen(path, "wb"));
  if (!f.f) return EHYB_ERR_IO;
  bool ok = std::fwrite(&h, sizeof(h), 1, f.f) == 1;
  for_each_array(*src, [&](const auto& v) {
    if (ok && !v.empty()) ok = std::fwrite(v.data(), sizeof(v[0]), v.size(), f.f) == v.size();
  });
  if (std::fclose(f.f) != 0) ok = false;
  f.f = nullptr;
  return ok ? EHYB_OK : EHYB_ERR_IO;
}

extern "C" ehyb_status_t ehyb_plan_load(const char* path, const ehyb_options_t* opt_in, void* stream,
                                        ehyb_plan_t* out) {
  if (!path || !out) return EHYB_ERR_INVALID_ARG;
  *out = nullptr;
  ehyb_options_t opt;
  if (opt_in) opt = *opt_in;
  else ehyb_options_default(&opt);
  auto pow2_or_zero = [](int32_t v) { return v == 0 || (v >= 1 && v <= 32 && (v & (v - 1)) == 0); };
  if (opt.lowp < 0 || opt.lowp > 2 || !pow2_or_zero(opt.er_tpr) || opt.num_sms < 0 || opt.wait_timeout_ns < 0 ||
      (opt.lowp_group != 0 && opt.lowp_group != 1 && opt.lowp_group != 4) ||
      (opt.block_threads != 0 && (opt.block_threads < 32 || opt.block_threads > 1024 || opt.block_threads % 32)))
    return EHYB_ERR_INVALID_ARG;
  File f(std::fopen(path, "rb"));
  if (!f.f) return EHYB_ERR_IO;
  FileHeader h;
  if (std::fread(&h, sizeof(h), 1, f.f) != 1) return EHYB_ERR_IO;
  if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion || h.header_bytes != sizeof(FileHeader))
    return EHYB_ERR_IO;
  for (int i = 0; i < kArrays; ++i)
    if (h.len[i] < 0 || h.len[i] > ((int64_t)1 << 40)) return EHYB_ERR_IO;
  std::unique_ptr<ehyb_plan_s> P;
  try {
    P.reset(new ehyb_plan_s());
  } catch (const std::bad_alloc&) {
    return EHYB_ERR_OOM;
  }
  HostPlan& H = P->host;
  H.n = h.n;
  H.nnz = h.nnz;
  H.nparts = h.nparts;
  H.nslices = h.nslices;
  H.tpr = h.tpr;
  H.slice_rows = h.slice_rows;
  H.er_layout = h.er_layout;
  H.max_part_rows = h.max_part_rows;
  H.er_nnz = h.er_nnz;
  H.ell_nnz = h.ell_nnz;
  int i = 0;
  bool ok = true;
  Fnv fnv;
  try {
    for_each_array(H, [&](auto& v) {
      const int64_t len = h.len[i++];
      if (!ok) return;
      v.resize((size_t)len);
      if (len) ok = std::fread(v.data(), sizeof(v[0]), (size_t)len, f.f) == (size_t)len;
      if (ok) fnv.add(v.data(), (size_t)len * sizeof(v[0]));
    });
  } catch (const std::bad_alloc&) {
    return EHYB_ERR_OOM;
  }
  if (!ok || fnv.done() != h.checksum || !valid(H, h)) return EHYB_ERR_IO;
  H.old_to_new.assign((size_t)H.n, 0);
  for (int64_t r = 0; r < H.n; ++r) H.old_to_new[(size_t)H.new_to_old[(size_t)r]] = (int32_t)r;
  make_lowp_copies(H, opt.lowp, opt.lowp_group);

  int dev = 0, sms = 0, optin = 0;
  if (opt.host_only) {
    sms = opt.num_sms > 0 ? opt.num_sms : 152;
  } else {
    ehyb_status_t st = device_query(&dev, &sms, &optin);
    if (st != EHYB_OK) return st;
    if ((int64_t)(H.max_part_rows + 2) * 8 > (int64_t)optin - 1024) return EHYB_ERR_TOO_LARGE;
  }
  ehyb_status_t st = plan_finalize(P, opt, dev, sms, stream, out);
  if (st != EHYB_OK) return st;
  (*out)->tuner_path = h.tuner_path;
  (*out)->ell_width_cap = h.ell_width_cap;
  return EHYB_OK;
}
