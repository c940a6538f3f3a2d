// Forward checkpoint and resume of a propagation (not part of the method): the orbitals in the
// Loewdin basis, the time and step count, and the density-derived state the next step starts
// from (rho_n, v_H, v_xc at the quadrature points, the nodal Hartree potential that warm-starts
// the iterative solver, and the previous step's v_H + v_xc of the extrapolated scheme), so that
// a resumed run takes the same steps as an uninterrupted one.
//
// File layout (host byte order, written by this library only):
//   header (struct CkptHeader below): magic "EFECKPT1", version, the sizes the payload was
//   written for, t, step, which optional parts are present, the adaptive Krylov sub-step count,
//   the payload's byte count and its 64-bit FNV-1a checksum;
//   payload: psi_bar [n_dof][n_cols] complex128, then with the state: rho, v_H, v_xc
//   [batch][n_cells][n_q] and phi [n_h][batch], then with the history: v_Hxc of the previous
//   step [batch][n_cells][n_q].
// A file is written to `path`.tmp and renamed, so an interrupted write leaves the previous
// checkpoint in place.  Reading checks the magic, version, sizes, payload length and checksum
// before anything is copied to the device.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "efe_internal.h"

namespace efe {
namespace {

struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t n_dof, n_cols, batch, n_cells, n_q, n_h;
  double t;
  int64_t step;
  int32_t has_state, has_prev;
  int32_t substeps;            // adaptive Krylov sub-steps of the next exponential (0: not recorded)
  int32_t reserved;
  uint64_t payload_bytes;
  uint64_t checksum;
};
constexpr char kMagic[8] = {'E', 'F', 'E', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kVersion = 1;

// Fowler-Noll-Vo 1a, 64 bits
uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

size_t payload_doubles(const CkptHeader& h) {
  const size_t nq = (size_t)h.batch * h.n_cells * h.n_q;
  size_t n = (size_t)h.n_dof * h.n_cols * 2;
  if (h.has_state) n += 3 * nq + (size_t)h.n_h * h.batch;
  if (h.has_prev) n += nq;
  return n;
}

// Reads and validates a checkpoint: header, payload length, checksum.  On success `payload`
// holds the doubles in file order.
bool read_file(const char* path, CkptHeader& h, std::vector<double>& payload, std::string& why) {
  FILE* f = fopen(path, "rb");
  if (!f) {
    why = std::string("cannot open ") + path;
    return false;
  }
  bool ok = fread(&h, sizeof h, 1, f) == 1;
  if (!ok) why = "file shorter than a checkpoint header";
  if (ok && (memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion || h.header_bytes != sizeof h)) {
    ok = false;
    why = "not a checkpoint of this version (magic, version or header size)";
  }
  if (ok && (h.n_dof < 1 || h.n_cols < 1 || h.batch < 1 || h.n_cells < 1 || h.n_q < 1 || h.n_h < 1 ||
             (h.has_state != 0 && h.has_state != 1) || (h.has_prev != 0 && h.has_prev != 1) ||
             h.substeps < 0 || h.substeps > 64 ||
             h.payload_bytes != payload_doubles(h) * sizeof(double))) {
    ok = false;
    why = "inconsistent checkpoint header";
  }
  if (ok) {
    payload.resize(payload_doubles(h));
    if (fread(payload.data(), sizeof(double), payload.size(), f) != payload.size()) {
      ok = false;
      why = "checkpoint payload truncated";
    } else if (fgetc(f) != EOF) {
      ok = false;
      why = "trailing bytes after the checkpoint payload";
    } else if (fnv1a(payload.data(), payload.size() * sizeof(double)) != h.checksum) {
      ok = false;
      why = "checkpoint checksum mismatch (corrupt file)";
    }
  }
  fclose(f);
  return ok;
}

thread_local std::string g_ckpt_err;

}  // namespace

// Host writer shared by efe_checkpoint_write_host and efe_checkpoint_save.
static efe_status write_file(const char* path, const CkptHeader& h0, const std::vector<const double*>& parts,
                             const std::vector<size_t>& counts, std::string& why) {
  CkptHeader h = h0;
  memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof h;
  size_t total = 0;
  uint64_t cs = 1469598103934665603ull;
  for (size_t i = 0; i < parts.size(); ++i) {
    total += counts[i];
    cs = fnv1a(parts[i], counts[i] * sizeof(double), cs);
  }
  if (total != payload_doubles(h)) {
    why = "checkpoint parts do not match the header";
    return EFE_ERR_ARG;
  }
  h.payload_bytes = total * sizeof(double);
  h.checksum = cs;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) {
    why = "cannot create " + tmp;
    return EFE_ERR_ARG;
  }
  bool ok = fwrite(&h, sizeof h, 1, f) == 1;
  for (size_t i = 0; ok && i < parts.size(); ++i) ok = fwrite(parts[i], sizeof(double), counts[i], f) == counts[i];
  ok = (fclose(f) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    why = std::string("writing ") + path + " failed";
    return EFE_ERR_ARG;
  }
  return EFE_OK;
}

}  // namespace efe

using namespace efe;

extern "C" {

const char* efe_checkpoint_last_error(void) { return g_ckpt_err.c_str(); }

static efe_status write_host_impl(const char* path, const int64_t* sizes, double t, int64_t step, int32_t substeps,
                                  const double* psi_host, const double* rho_host, const double* vH_host,
                                  const double* vxc_host, const double* phi_host, const double* vprev_host) {
  g_ckpt_err.clear();
  if (!path || !sizes || !psi_host) {
    g_ckpt_err = "null path, sizes or orbitals";
    return EFE_ERR_ARG;
  }
  const bool state = rho_host && vH_host && vxc_host && phi_host;
  if ((rho_host || vH_host || vxc_host || phi_host) && !state) {
    g_ckpt_err = "the state needs rho, v_H, v_xc and phi together";
    return EFE_ERR_ARG;
  }
  if (vprev_host && !state) {
    g_ckpt_err = "the previous potential needs the state";
    return EFE_ERR_ARG;
  }
  CkptHeader h{};
  h.n_dof = sizes[0];
  h.n_cols = sizes[1];
  h.batch = sizes[2];
  h.n_cells = sizes[3];
  h.n_q = sizes[4];
  h.n_h = sizes[5];
  h.t = t;
  h.step = step;
  h.has_state = state ? 1 : 0;
  h.has_prev = vprev_host ? 1 : 0;
  h.substeps = substeps;
  for (int i = 0; i < 6; ++i)
    if (sizes[i] < 1) {
      g_ckpt_err = "sizes must be >= 1";
      return EFE_ERR_ARG;
    }
  const size_t nq = (size_t)h.batch * h.n_cells * h.n_q;
  std::vector<const double*> parts{psi_host};
  std::vector<size_t> counts{(size_t)h.n_dof * h.n_cols * 2};
  if (state) {
    parts.insert(parts.end(), {rho_host, vH_host, vxc_host, phi_host});
    counts.insert(counts.end(), {nq, nq, nq, (size_t)h.n_h * h.batch});
  }
  if (vprev_host) {
    parts.push_back(vprev_host);
    counts.push_back(nq);
  }
  return write_file(path, h, parts, counts, g_ckpt_err);
}

efe_status efe_checkpoint_write_host(const char* path, const int64_t* sizes, double t, int64_t step,
                                     const double* psi_host, const double* rho_host, const double* vH_host,
                                     const double* vxc_host, const double* phi_host, const double* vprev_host) {
  return write_host_impl(path, sizes, t, step, 0, psi_host, rho_host, vH_host, vxc_host, phi_host, vprev_host);
}

efe_status efe_checkpoint_inspect(const char* path, int64_t* sizes, double* t, int64_t* step, int32_t* has_state,
                                  int32_t* has_prev) {
  g_ckpt_err.clear();
  if (!path) {
    g_ckpt_err = "efe_checkpoint_inspect: path is NULL";
    return EFE_ERR_ARG;
  }
  CkptHeader h{};
  std::vector<double> payload;
  if (!read_file(path, h, payload, g_ckpt_err)) return EFE_ERR_ARG;
  if (sizes) {
    const int64_t s[6] = {h.n_dof, h.n_cols, h.batch, h.n_cells, h.n_q, h.n_h};
    memcpy(sizes, s, sizeof s);
  }
  if (t) *t = h.t;
  if (step) *step = h.step;
  if (has_state) *has_state = h.has_state;
  if (has_prev) *has_prev = h.has_prev;
  return EFE_OK;
}

efe_status efe_checkpoint_save(efe_ctx* ctx, const char* path, const double* psi_bar_dev, double t, int64_t step,
                               void* stream) {
  if (!ctx) return EFE_ERR_ARG;
  Ctx& c = ctx->c;
  c.err.clear();
  if (!path || !psi_bar_dev) {
    c.err = "efe_checkpoint_save: null path or orbitals";
    return EFE_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long C = (long long)c.n_orb * c.batch;
  const size_t nq = (size_t)c.batch * c.nc * c.nq;
  std::vector<double> psi((size_t)c.n_dof * C * 2), rho, vH, vxc, phi, vprev;
  cudaError_t e = cudaMemcpyAsync(psi.data(), psi_bar_dev, sizeof(double) * psi.size(), cudaMemcpyDeviceToHost, s);
  const bool state = c.state_valid && c.d_rho;
  const bool prev = state && c.has_prev && c.d_vprev;
  if (e == cudaSuccess && state) {
    rho.resize(nq);
    vH.resize(nq);
    vxc.resize(nq);
    phi.resize((size_t)c.n_h * c.batch);
    e = cudaMemcpyAsync(rho.data(), c.d_rho, sizeof(double) * nq, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vH.data(), c.d_vH, sizeof(double) * nq, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vxc.data(), c.d_vxc, sizeof(double) * nq, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(phi.data(), c.d_phi, sizeof(double) * phi.size(), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess && prev) {
    vprev.resize(nq);
    e = cudaMemcpyAsync(vprev.data(), c.d_vprev, sizeof(double) * nq, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    c.err = std::string("efe_checkpoint_save: ") + cudaGetErrorString(e);
    return EFE_ERR_CUDA;
  }
  const int64_t sizes[6] = {c.n_dof, C, c.batch, c.nc, c.nq, c.n_h};
  const efe_status st = write_host_impl(path, sizes, t, step, c.substeps_opt == 0 ? c.substeps_cur : 0, psi.data(),
                                       state ? rho.data() : nullptr, state ? vH.data() : nullptr,
                                       state ? vxc.data() : nullptr, state ? phi.data() : nullptr,
                                       prev ? vprev.data() : nullptr);
  if (st != EFE_OK) c.err = "efe_checkpoint_save: " + g_ckpt_err;
  return st;
}

efe_status efe_checkpoint_load(efe_ctx* ctx, const char* path, double* psi_bar_dev, double* t_host,
                               int64_t* step_host, void* stream) {
  if (!ctx) return EFE_ERR_ARG;
  Ctx& c = ctx->c;
  c.err.clear();
  if (!path || !psi_bar_dev) {
    c.err = "efe_checkpoint_load: null path or orbitals";
    return EFE_ERR_ARG;
  }
  CkptHeader h{};
  std::vector<double> payload;
  std::string why;
  if (!read_file(path, h, payload, why)) {
    c.err = "efe_checkpoint_load: " + why;
    return EFE_ERR_ARG;
  }
  const long long C = (long long)c.n_orb * c.batch;
  if (h.n_dof != c.n_dof || h.n_cols != C || h.batch != c.batch || h.n_cells != c.nc || h.n_q != c.nq ||
      h.n_h != c.n_h) {
    c.err = "efe_checkpoint_load: the checkpoint was written for other sizes (n_dof, orbitals, batch or mesh)";
    return EFE_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t nq = (size_t)c.batch * c.nc * c.nq, npsi = (size_t)c.n_dof * C * 2;
  if (h.has_state && !c.d_rho) {   // the context's state buffers (allocated at its first step otherwise)
    const size_t nqb = nq;
    if (cudaMalloc(&c.d_rho, sizeof(double) * nqb) != cudaSuccess ||
        cudaMalloc(&c.d_vprev, sizeof(double) * nqb) != cudaSuccess ||
        cudaMalloc(&c.d_vH, sizeof(double) * nqb) != cudaSuccess ||
        cudaMalloc(&c.d_vxc, sizeof(double) * nqb) != cudaSuccess ||
        cudaMalloc(&c.d_rho2, sizeof(double) * nqb) != cudaSuccess ||
        cudaMalloc(&c.d_v, sizeof(double) * nqb) != cudaSuccess ||
        cudaMalloc(&c.d_cg, sizeof(double) * ((size_t)6 * c.n_h * c.batch + 5 * c.batch)) != cudaSuccess ||
        cudaMalloc(&c.d_phi, sizeof(double) * (size_t)c.n_h * c.batch) != cudaSuccess) {
      c.err = "efe_checkpoint_load: out of device memory for the state";
      return EFE_ERR_NOMEM;
    }
  }
  const double* p = payload.data();
  cudaError_t e = cudaMemcpyAsync(psi_bar_dev, p, sizeof(double) * npsi, cudaMemcpyHostToDevice, s);
  p += npsi;
  if (h.has_state) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_rho, p, sizeof(double) * nq, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_vH, p + nq, sizeof(double) * nq, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_vxc, p + 2 * nq, sizeof(double) * nq, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c.d_phi, p + 3 * nq, sizeof(double) * (size_t)c.n_h * c.batch, cudaMemcpyHostToDevice, s);
    p += 3 * nq + (size_t)c.n_h * c.batch;
  }
  if (h.has_prev && e == cudaSuccess) e = cudaMemcpyAsync(c.d_vprev, p, sizeof(double) * nq, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host payload must outlive the copies
  if (e != cudaSuccess) {
    c.err = std::string("efe_checkpoint_load: ") + cudaGetErrorString(e);
    return EFE_ERR_CUDA;
  }
  c.state_valid = h.has_state != 0;
  c.has_prev = h.has_prev != 0;
  if (c.substeps_opt == 0 && h.substeps > 0) c.substeps_cur = h.substeps;
  if (t_host) *t_host = h.t;
  if (step_host) *step_host = h.step;
  return EFE_OK;
}

}  // extern "C"
