"""The C ABI used from C (no Python in the client): tests/helpers/c_abi_client.c compiles and
links against include/abp.h and libabp.so on the host (no GPU needed); on a GPU its moments are
the exact bits the Python binding gets for the same batch."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "helpers", "c_abi_client.c")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    from paper_1104_2499_gb300 import build as B

    try:
        B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available to build libabp.so")
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    lib = B.build()
    exe = str(tmp_path_factory.mktemp("cabi") / "c_abi_client")
    subprocess.run(["gcc", "-std=c11", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), SRC, "-o", exe,
                    "-L", os.path.dirname(lib), "-labp", "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    return exe


def test_c_client_compiles_and_links(client):
    assert os.access(client, os.X_OK)


@pytest.mark.gpu
def test_c_client_gets_the_bindings_bits(client):
    torch = pytest.importorskip("torch")
    from paper_1104_2499_gb300 import abp as A
    from paper_1104_2499_gb300 import workloads as W

    out = subprocess.run([client, "11"], capture_output=True, text=True, check=True).stdout.strip().splitlines()
    got = np.array([[float.fromhex(v) for v in line.split()[2:10]] for line in out])
    hist = [int(line.split()[-1]) for line in out]
    sets = [W.params(q=1.0, D=0.1, asym=0.25), W.params(q=2.0, F0=-0.2, D=0.3, asym=0.1)]
    w = W.Workload(name="cabi", sets=sets, n_traj=[1000, 517], n_steps=[2000, 1500], dt=1e-3, seed=11, v0_mode=1,
                   hist_x_bins=16)
    with A.Ensemble(w, particles_per_thread=2, schedule=1) as ens:
        ens.run()
        ref = ens.results(host=True)["moments"].numpy()
    assert np.array_equal(got, ref), (got, ref)
    assert hist == [1000, 517]
    assert torch.cuda.is_available()
