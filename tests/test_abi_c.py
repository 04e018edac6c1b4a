"""include/tdgrad.h is a plain C interface: a C99 program (strict, -pedantic,
warnings as errors) compiles against it, links libtdgrad.so and uses the
host-side calls (options, status strings, argument checks, the router's
handle and file).  No compute call is made, so this runs without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <string.h>
#include "tdgrad.h"

int main(int argc, char **argv)
{
    tg_options o;
    tg_router *r = NULL, *r2 = NULL;
    tg_basis *b = (tg_basis *)&o;
    float p[2048], p2[2048], mu[16], sd[16], cal[3];
    double xyz[3] = {0.0, 0.0, 0.0}, ex[1] = {-1.0}, co[1] = {1.0};
    int atom[1] = {0}, l[1] = {0}, np[1] = {1}, n, k, rc;
    const char *path = argc > 1 ? argv[1] : "r.bin";

    tg_options_default(&o);
    printf("defaults %g %d %d %g\n", o.screen_tol, o.precision, o.nranks, o.mixed_tol);
    for (k = 0; k >= -6; --k) printf("status %d %s\n", k, tg_strerror(k));
    /* a non-positive exponent is refused before any device call; *out is cleared */
    rc = tg_basis_create(1, xyz, 1, atom, l, np, ex, co, &b);
    printf("basis_bad_exponent %d %d\n", rc, b == NULL);
    l[0] = 3;
    ex[0] = 1.0;
    printf("basis_f_shell %d\n", tg_basis_create(1, xyz, 1, atom, l, np, ex, co, &b));
    n = tg_router_nparam();
    printf("nparam %d\n", n);
    if (n > 2048) return 2;
    if (tg_router_create(42ULL, &r) != TG_OK) return 3;
    for (k = 0; k < 16; ++k) {
        mu[k] = 0.1f * (float)k;
        sd[k] = 1.0f + (float)k;
    }
    cal[0] = -0.25f;
    cal[1] = 2e-6f;
    cal[2] = 1.0f;
    if (tg_router_set(r, NULL, mu, sd, cal) != TG_OK) return 4;
    sd[3] = -1.0f;
    printf("set_bad_sd %d\n", tg_router_set(r, NULL, NULL, sd, NULL));
    if (tg_router_save(r, path) != TG_OK) return 5;
    if (tg_router_load(path, &r2) != TG_OK) return 6;
    tg_router_get(r, p, NULL, NULL, NULL);
    tg_router_get(r2, p2, mu, sd, cal);
    printf("roundtrip %d %g %g %g %g\n", memcmp(p, p2, sizeof(float) * (size_t)n) == 0, mu[5], sd[3], cal[0],
           cal[2]);
    tg_router_destroy(r);
    tg_router_destroy(r2);
    printf("load_missing %d\n", tg_router_load("/nonexistent/router.bin", &r2));
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not found")
def test_header_is_plain_c_and_links(tmp_path):
    from paper_2407_16586_gb300 import build
    lib = build.build()
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L" + libdir, "-ltdgrad", "-Wl,-rpath," + libdir, "-lm"])
    out = subprocess.run([str(exe), str(tmp_path / "r.bin")], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = dict(line.split(" ", 1) for line in out.stdout.strip().splitlines() if not line.startswith("status"))
    assert lines["defaults"] == "1e-10 0 1 1e-06"
    status = [line for line in out.stdout.splitlines() if line.startswith("status")]
    assert len(status) == 7 and status[0] == "status 0 ok" and status[1] == "status -1 invalid argument"
    assert lines["basis_bad_exponent"] == "-1 1"
    assert lines["basis_f_shell"] == "-2"
    assert lines["nparam"] == "1633"
    assert lines["set_bad_sd"] == "-1"
    assert lines["roundtrip"] == "1 0.5 4 -0.25 1"
    assert lines["load_missing"] == "-6"
