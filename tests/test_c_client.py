"""The C ABI from a plain C program (tests/c_client/lagflux_client.c),
compiled with gcc against include/lagflux.h and linked to the library."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB_DIR = os.path.join(ROOT, "paper_1607_08710_gb300")


@pytest.fixture(scope="module")
def client():
    if not os.path.exists(os.path.join(LIB_DIR, "liblagflux.so")):
        pytest.skip("liblagflux.so not built")
    out = os.path.join(tempfile.mkdtemp(prefix="lagflux_client_"), "lagflux_client")
    subprocess.run(["gcc", "-std=c11", "-O1", "-Wall", "-Werror", "-D_DEFAULT_SOURCE",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_client", "lagflux_client.c"),
                    "-L", LIB_DIR, "-llagflux", "-Wl,-rpath," + LIB_DIR, "-lm", "-o", out], check=True)
    return out


def test_c_client_abi_without_gpu(client):
    r = subprocess.run([client, "abi"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.gpu
def test_c_client_runs_on_gpu(client):
    r = subprocess.run([client, "run"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "sums conserved" in r.stdout
