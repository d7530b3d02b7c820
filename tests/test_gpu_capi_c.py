"""The C ABI used from C: a program compiled with the system C compiler against include/cbgmres.h
and linked with libcbgmres.so and the CUDA runtime runs cbgmres_create -> cbgmres_solve ->
cbgmres_destroy on the 64x64 convection-diffusion system (wind (1, 0.5), Peclet 10, b = A x_true,
restart 50, tol 1e-10, x0 = 0) through device buffers it prepares itself. Its result is checked
against the oracle's solve stored in tests/golden/solve_c1_<format>.json (written by
tests/golden/make_solve_references.py): iterations within 2%, the same second-pass and breakdown
counts, and the solution at the stored sample of indices within 1e-8 (relative)."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime.h>
#include "cbgmres.h"

static void* slurp(const char* path, size_t bytes) {
  FILE* f = fopen(path, "rb");
  if (!f) return NULL;
  void* p = malloc(bytes ? bytes : 1);
  size_t got = fread(p, 1, bytes, f);
  fclose(f);
  if (got != bytes) { free(p); return NULL; }
  return p;
}

#define CUDA_OK(call) do { if ((call) != cudaSuccess) { fprintf(stderr, "cuda failure: %s\n", #call); return 3; } } while (0)

int main(int argc, char** argv) {
  if (argc != 8) return 2;
  const int32_t n = atoi(argv[1]);
  const int64_t nnz = atoll(argv[2]);
  const char* dir = argv[3];
  const int32_t fmt = atoi(argv[4]), bits = atoi(argv[5]), cycle = atoi(argv[6]);
  char path[4096];
  snprintf(path, sizeof path, "%s/row_ptr.bin", dir);
  int32_t* rp = slurp(path, sizeof(int32_t) * (n + 1));
  snprintf(path, sizeof path, "%s/col.bin", dir);
  int32_t* col = slurp(path, sizeof(int32_t) * nnz);
  snprintf(path, sizeof path, "%s/vals.bin", dir);
  double* vals = slurp(path, sizeof(double) * nnz);
  snprintf(path, sizeof path, "%s/b.bin", dir);
  double* b = slurp(path, sizeof(double) * n);
  if (!rp || !col || !vals || !b) return 4;
  int32_t *d_rp, *d_col;
  double *d_vals, *d_b, *d_x;
  CUDA_OK(cudaMalloc((void**)&d_rp, sizeof(int32_t) * (n + 1)));
  CUDA_OK(cudaMalloc((void**)&d_col, sizeof(int32_t) * nnz));
  CUDA_OK(cudaMalloc((void**)&d_vals, sizeof(double) * nnz));
  CUDA_OK(cudaMalloc((void**)&d_b, sizeof(double) * n));
  CUDA_OK(cudaMalloc((void**)&d_x, sizeof(double) * n));
  CUDA_OK(cudaMemcpy(d_rp, rp, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
  CUDA_OK(cudaMemcpy(d_col, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
  CUDA_OK(cudaMemcpy(d_vals, vals, sizeof(double) * nnz, cudaMemcpyHostToDevice));
  CUDA_OK(cudaMemcpy(d_b, b, sizeof(double) * n, cudaMemcpyHostToDevice));
  CUDA_OK(cudaMemset(d_x, 0, sizeof(double) * n));

  cbg_opts o;
  if (cbg_opts_default(&o) != CBG_OK) return 5;
  o.restart = 50;
  o.fmt = fmt;
  o.frsz2_bits = bits;
  o.tol = 1e-10;
  o.cycle = cycle;
  cbg_ctx* ctx = NULL;
  int st = cbgmres_create(&ctx, n, nnz, d_rp, d_col, d_vals, &o, NULL);
  if (st != CBG_OK) {
    fprintf(stderr, "create: %d %s\n", st, cbgmres_last_error());
    return 6;
  }
  cbg_result r;
  st = cbgmres_solve(ctx, d_b, d_x, &r);
  double* x = malloc(sizeof(double) * n);
  CUDA_OK(cudaMemcpy(x, d_x, sizeof(double) * n, cudaMemcpyDeviceToHost));
  const int32_t cluster = cbgmres_cycle_cluster(ctx);
  if (cbgmres_destroy(ctx) != CBG_OK) return 7;
  snprintf(path, sizeof path, "%s/x.bin", dir);
  FILE* f = fopen(path, "wb");
  if (!f || fwrite(x, sizeof(double), n, f) != (size_t)n) return 8;
  fclose(f);
  printf("%d %lld %lld %lld %lld %d %.17g %d\n", st, (long long)r.iters, (long long)r.restarts, (long long)r.reorths,
         (long long)r.breakdowns, r.converged, r.true_rrn, cluster);
  cudaFree(d_rp); cudaFree(d_col); cudaFree(d_vals); cudaFree(d_b); cudaFree(d_x);
  free(rp); free(col); free(vals); free(b); free(x);
  return 0;
}
"""


def cuda_dirs():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    inc = os.path.join(home, "include")
    libs = [os.path.join(home, d) for d in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib")]
    lib = next((d for d in libs if os.path.exists(os.path.join(d, "libcudart.so"))), None)
    return inc, lib


@pytest.fixture(scope="module")
def program(cbg, tmp_path_factory):
    cc = shutil.which("cc") or shutil.which("gcc")
    inc, cudalib = cuda_dirs()
    if cc is None or cudalib is None:
        pytest.skip("no C compiler or CUDA runtime library")
    d = tmp_path_factory.mktemp("capi_c")
    src = d / "solve.c"
    src.write_text(PROGRAM)
    exe = d / "solve"
    libdir = os.path.dirname(cbg.library_path())
    subprocess.run([cc, "-std=c11", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I", inc,
                    str(src), "-o", str(exe), "-L", libdir, "-lcbgmres", "-L", cudalib, "-lcudart",
                    f"-Wl,-rpath,{libdir}:{cudalib}"], check=True)
    return exe


@pytest.mark.parametrize("cycle", [0, 1])
@pytest.mark.parametrize("fmt,bits,name", [(0, 32, "fp64"), (4, 32, "frsz2_32"), (1, 32, "fp32"), (4, 16, "frsz2_16")])
def test_c_program_solves_c1(program, tmp_path, fmt, bits, name, cycle):
    with open(os.path.join(ROOT, "tests", "golden", f"solve_c1_{name}.json")) as f:
        ref = json.load(f)
    A = workloads.convdiff(64, 2, (1.0, 0.5), 10.0)
    rp, col, vals = A.numpy()
    import oracle

    b = oracle.spmv(rp, col, vals, workloads.uniform_vector(A.n, 0).numpy())
    rp.astype(np.int32).tofile(tmp_path / "row_ptr.bin")
    col.astype(np.int32).tofile(tmp_path / "col.bin")
    vals.astype(np.float64).tofile(tmp_path / "vals.bin")
    b.tofile(tmp_path / "b.bin")
    out = subprocess.run([str(program), str(A.n), str(A.nnz), str(tmp_path), str(fmt), str(bits), str(cycle),
                          "-"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    st, iters, restarts, reorths, breakdowns, converged, rrn, cluster = out.stdout.split()
    assert int(st) == 0 and int(converged) == 1 and float(rrn) <= 1e-10
    assert (int(cluster) > 0) == (cycle == 0)
    assert abs(int(iters) - ref["iters"]) <= max(1, 0.02 * ref["iters"]), (iters, ref["iters"])
    assert int(breakdowns) == ref["breakdowns"]
    assert abs(int(reorths) - ref["reorths"]) <= abs(int(iters) - ref["iters"]), (reorths, ref["reorths"])
    x = np.fromfile(tmp_path / "x.bin", dtype=np.float64)
    idx = np.array(ref["sample_index"])
    xo = np.array([float.fromhex(v) for v in ref["sample_x"]])
    assert np.linalg.norm(x[idx] - xo) / np.linalg.norm(xo) <= 1e-8
