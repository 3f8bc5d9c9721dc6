"""The GPU noise stream against cuRAND's Philox4x32-10 (NVIDIA's implementation of the
same published generator, run as a library): block m of trajectory t under seed s must be
the state cuRAND reaches with curand_init(s, t, 4 m).  An independent check of the kernels'
Philox beside the oracle's (which is pinned to ATen's host engine)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_kat(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    so = str(tmp_path_factory.mktemp("curand") / "libcurand_kat.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    os.path.join(HERE, "helpers", "curand_philox_kat.cu"), "-o", so], check=True)
    L = C.CDLL(so)
    L.curand_philox_blocks.argtypes = [C.c_uint64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    L.curand_philox_blocks.restype = C.c_int
    return L


def test_philox_blocks_match_curand(curand_kat):
    from paper_1104_2499_gb300 import abp as A
    from paper_1104_2499_gb300 import build as B

    B.build()
    A.lib()
    rng = np.random.default_rng(11)
    n = 1 << 14
    t = rng.integers(0, 2**40, n, dtype=np.uint64)
    m = rng.integers(0, 2**30, n, dtype=np.uint64)  # 4 m stays a valid 64-bit offset
    t[:3] = [0, 1, 2**40 - 1]
    m[:3] = [0, 1, 2**30 - 1]
    for seed in (0, 1, 0x0123456789ABCDEF):
        t_d = torch.from_numpy(t.view(np.int64)).cuda()
        m_d = torch.from_numpy(m.view(np.int64)).cuda()
        ours = torch.empty((n, 4), dtype=torch.int32, device="cuda")
        ref = torch.empty((n, 4), dtype=torch.int32, device="cuda")
        A.abp_philox(seed, t_d, m_d, ours)
        torch.cuda.synchronize()
        assert curand_kat.curand_philox_blocks(seed, t_d.data_ptr(), m_d.data_ptr(), n, ref.data_ptr()) == 0
        np.testing.assert_array_equal(ours.cpu().numpy(), ref.cpu().numpy())
