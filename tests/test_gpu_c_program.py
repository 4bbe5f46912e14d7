"""The boundary from C on the GPU: a C99 program linked against libaidw.so runs interpolations
with host arrays, with no Python in the loop. It creates a dataset, calls aidw_interpolate in
FP32 (with alpha and kNN outputs) and in FP64, serves the FP32 request again through
aidw_submit + aidw_wait, and writes every output to a file; the test compares them with the
FP64 oracle: both FP32 results within 1e-5 (the served one runs through the batch kernel) and
the direct call's kNN lists equal up to FP32 distance ties; FP64 within 1e-12 with identical kNN
lists."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw, build, workloads
from parity import TOL_F32, TOL_F64, knn_mismatch, oracle_for, rel_err

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "aidw.h"

static int read_all(const char *path, void *buf, size_t bytes)
{
    FILE *f = fopen(path, "rb");
    if (!f)
        return -1;
    size_t got = fread(buf, 1, bytes, f);
    fclose(f);
    return got == bytes ? 0 : -1;
}

static int write_all(const char *path, const void *buf, size_t bytes)
{
    FILE *f = fopen(path, "wb");
    if (!f)
        return -1;
    size_t put = fwrite(buf, 1, bytes, f);
    fclose(f);
    return put == bytes ? 0 : -1;
}

/* argv: dir n m k area. Inputs dir/x dir/y dir/z (n doubles), dir/qx dir/qy (m doubles). */
int main(int argc, char **argv)
{
    if (argc != 6)
        return 2;
    const char *dir = argv[1];
    const int64_t n = atoll(argv[2]), m = atoll(argv[3]);
    const int k = atoi(argv[4]);
    const double area = atof(argv[5]);
    char path[4096];
    double *x = malloc(sizeof(double) * n), *y = malloc(sizeof(double) * n);
    double *z = malloc(sizeof(double) * n);
    double *qx = malloc(sizeof(double) * m), *qy = malloc(sizeof(double) * m);
    float *fqx = malloc(sizeof(float) * m), *fqy = malloc(sizeof(float) * m);
    float *z32 = malloc(sizeof(float) * m), *z32s = malloc(sizeof(float) * m);
    float *a32 = malloc(sizeof(float) * m);
    int32_t *knn32 = malloc(sizeof(int32_t) * m * k), *knn64 = malloc(sizeof(int32_t) * m * k);
    double *z64 = malloc(sizeof(double) * m);
    if (!x || !y || !z || !qx || !qy || !fqx || !fqy || !z32 || !z32s || !a32 || !knn32 ||
        !knn64 || !z64)
        return 3;
    const char *names[5] = {"x", "y", "z", "qx", "qy"};
    double *arrays[5] = {x, y, z, qx, qy};
    for (int i = 0; i < 5; ++i) {
        snprintf(path, sizeof path, "%s/%s", dir, names[i]);
        if (read_all(path, arrays[i], sizeof(double) * (i < 3 ? n : m)))
            return 4;
    }
    for (int64_t j = 0; j < m; ++j) {
        fqx[j] = (float)qx[j];
        fqy[j] = (float)qy[j];
    }

    aidw_ctx *ctx = NULL;
    int rc = aidw_init(&ctx, 0, 0);
    if (rc != AIDW_OK) {
        fprintf(stderr, "aidw_init: %s\n", aidw_status_string(rc));
        return 5;
    }
    aidw_dataset ds = 0;
    rc = aidw_create_dataset(ctx, x, y, z, n, area, AIDW_DTYPE_F64, &ds);
    if (rc != AIDW_OK) {
        fprintf(stderr, "aidw_create_dataset: %s\n", aidw_status_string(rc));
        return 6;
    }
    aidw_params p;
    aidw_params_default(&p);
    p.k = k;
    rc = aidw_interpolate(ctx, ds, fqx, fqy, m, &p, z32, a32, knn32, NULL);
    if (rc != AIDW_OK) {
        fprintf(stderr, "aidw_interpolate F32C: %s\n", aidw_status_string(rc));
        return 7;
    }
    aidw_request id = 0;
    rc = aidw_submit(ctx, ds, fqx, fqy, m, &p, z32s, NULL, NULL, &id);
    if (rc == AIDW_OK)
        rc = aidw_wait(ctx, id, 60000000);
    if (rc != AIDW_OK) {
        fprintf(stderr, "aidw_submit / aidw_wait: %s\n", aidw_status_string(rc));
        return 8;
    }
    aidw_release_request(ctx, id);
    p.precision = AIDW_F64;
    rc = aidw_interpolate(ctx, ds, qx, qy, m, &p, z64, NULL, knn64, NULL);
    if (rc != AIDW_OK) {
        fprintf(stderr, "aidw_interpolate F64: %s\n", aidw_status_string(rc));
        return 9;
    }
    if (aidw_check_device_errors(ctx) != AIDW_OK)
        return 10;
    aidw_destroy_dataset(ctx, ds);
    aidw_shutdown(ctx);

    const char *onames[6] = {"z32", "z32s", "a32", "knn32", "z64", "knn64"};
    const void *outs[6] = {z32, z32s, a32, knn32, z64, knn64};
    const size_t bytes[6] = {4 * (size_t)m, 4 * (size_t)m, 4 * (size_t)m, 4 * (size_t)(m * k),
                             8 * (size_t)m, 4 * (size_t)(m * k)};
    for (int i = 0; i < 6; ++i) {
        snprintf(path, sizeof path, "%s/%s.out", dir, onames[i]);
        if (write_all(path, outs[i], bytes[i]))
            return 11;
    }
    printf("ok\n");
    return 0;
}
"""


def test_c_program_interpolates_on_the_gpu(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    lib_path = build.build()
    src = tmp_path / "prog.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "prog"
    libdir = os.path.dirname(lib_path)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), lib_path,
                        f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    # One warp per query in FP32 and FP64 phase 1 (20,000 queries), clustered data.
    wl = workloads.small_case(301, 30000, 20000, k=10, pattern="clustered")
    for name in ("x", "y", "z", "qx", "qy"):
        np.ascontiguousarray(getattr(wl, name), dtype=np.float64).tofile(tmp_path / name)
    r = subprocess.run([str(exe), str(tmp_path), str(wl.n), str(wl.m), str(wl.k),
                        repr(wl.area)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    m, k = wl.m, wl.k
    z32 = np.fromfile(tmp_path / "z32.out", dtype=np.float32)
    z32s = np.fromfile(tmp_path / "z32s.out", dtype=np.float32)
    a32 = np.fromfile(tmp_path / "a32.out", dtype=np.float32)
    knn32 = np.fromfile(tmp_path / "knn32.out", dtype=np.int32).reshape(m, k)
    z64 = np.fromfile(tmp_path / "z64.out", dtype=np.float64)
    knn64 = np.fromfile(tmp_path / "knn64.out", dtype=np.int32).reshape(m, k)

    ref32, src32 = oracle_for(wl, aidw.F32C)
    assert rel_err(z32, ref32).max() <= TOL_F32
    assert not knn_mismatch(knn32, ref32, src32, aidw.F32C)
    assert np.abs(a32 - ref32["alpha"]).max() <= 2e-6 * 5.0
    # The served request runs through the batch kernel: its own tolerance against the oracle.
    assert rel_err(z32s, ref32).max() <= TOL_F32
    ref64, src64 = oracle_for(wl, aidw.F64)
    assert rel_err(z64, ref64).max() <= TOL_F64
    assert not knn_mismatch(knn64, ref64, src64, aidw.F64)
