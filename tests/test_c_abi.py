"""The boundary as C: include/aidw.h compiles as C99 (and as C++), and a C program linked against
libaidw.so runs the host-only parts of the ABI (status strings, parameter defaults, kernel-shape
validation, the tuning cache and its file) and gets clean errors from the device entry points
when no GPU is present."""
import os
import shutil
import subprocess

import pytest

from paper_1511_02186_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "aidw.h"

int main(int argc, char **argv)
{
    if (argc < 2)
        return 9;
    aidw_params p;
    aidw_params_default(&p);
    if (p.k != 10 || p.precision != AIDW_F32C || p.alpha[4] != 5.0 || p.r_max != 2.0)
        return 10;
    if (strcmp(aidw_status_string(AIDW_OK), aidw_status_string(AIDW_ERR_OOM)) == 0)
        return 11;
    aidw_tune_config c;
    if (aidw_tune_config_default(&c) != AIDW_OK || aidw_tune_config_check(&c) != AIDW_OK)
        return 12;
    c.tile_points = 300;
    if (aidw_tune_config_check(&c) != AIDW_ERR_INVALID_ARG)
        return 13;
    aidw_tune_config_default(&c);
    c.queries_per_thread = 8;
    if (aidw_tune_cache_put("c program key", &c, 1.5) != AIDW_OK)
        return 14;
    if (aidw_tune_cache_save(argv[1]) != AIDW_OK)
        return 15;
    aidw_tune_cache_clear();
    if (aidw_tune_cache_size() != 0 || aidw_tune_cache_load(argv[1]) != AIDW_OK)
        return 16;
    aidw_tune_config d;
    double ms = 0.0;
    if (aidw_tune_cache_get("c program key", &d, &ms) != AIDW_OK || d.queries_per_thread != 8 ||
        ms != 1.5)
        return 17;
    if (aidw_interpolate(NULL, 1, NULL, NULL, 0, &p, NULL, NULL, NULL, NULL) !=
        AIDW_ERR_INVALID_ARG)
        return 18;
    aidw_ctx *ctx = NULL;
    int rc = aidw_init(&ctx, 0, 0);
    printf("init %d\n", rc);
    if (rc == AIDW_OK)
        aidw_shutdown(ctx);
    printf("ok\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def lib_path():
    return build.build()


@pytest.mark.parametrize("compiler,flags", [("gcc", ["-std=c99", "-x", "c"]),
                                            ("g++", ["-std=c++17", "-x", "c++"])])
def test_c_program_against_the_library(tmp_path, lib_path, compiler, flags):
    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} not found")
    src = tmp_path / "prog.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "prog"
    libdir = os.path.dirname(lib_path)
    cmd = [compiler, *flags, "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           str(src), "-x", "none", lib_path, f"-Wl,-rpath,{libdir}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe), str(tmp_path / "cache.jsonl")], capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip().endswith("ok")
    assert (tmp_path / "cache.jsonl").read_text().count("c program key") == 1
