"""Failure detection on the GPU without a fault: the tensor-core engine's bounded
completion wait.

The mixed path's tensor-core block product completes on an mbarrier, and every
wait on it has an iteration limit.  A variant of the library built with
-DTTP_TC_LOOP_WAIT=0 makes the waits inside maxvol's visit loop give up without
polling (the products still run and complete; one poll would not do, since a
try-wait may itself suspend until the phase completes); the wait before the
tensor memory is released keeps its full limit.  The test checks that such a launch returns,
that every affected problem reports TT_ERR_NUMERIC with fail_step 6 and a NaN
price, and that the context stays usable: the regular library then prices the
same problems correctly in the same process.  No wait is left unbounded and no
GPU fault is involved."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2203_02804_gb300 import build, inputs

pytestmark = pytest.mark.gpu


def test_tensor_core_wait_gives_up_cleanly():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02804_gb300 import ttprice

    build.build()
    tmp = tempfile.mkdtemp(prefix="ttprice_wait_")
    lib_path = os.path.join(tmp, "libttprice_shortwait.so")
    subprocess.run([build.nvcc_path(), *build.ARCH, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                    "-DTTP_TC_LOOP_WAIT=0", "-I", build.INCLUDE, "-o", lib_path,
                    os.path.join(build.CSRC, "ttprice.cu")], check=True)
    short = ttprice.load_library(lib_path)
    ps = inputs.tuning_batch(6, 3, 32, 16)
    pr = ttprice.Pricer(max_d=3, max_n=32, max_rank=16, max_batch=len(ps), precision="mixed", engine="tc",
                        lib=short, use_torch_workspace=False, graph=False)
    rc, prices, diags = pr.evaluate(ps)
    pr.close()
    torch.cuda.synchronize()
    assert rc == ttprice.TT_ERR_NUMERIC
    assert all(d.status == ttprice.TT_ERR_NUMERIC and d.fail_step == 6 for d in diags)
    assert np.all(np.isnan(prices))
    # the context is intact: the regular build prices the same problems
    pr = ttprice.Pricer(max_d=3, max_n=32, max_rank=16, max_batch=len(ps), precision="mixed", engine="tc")
    rc, prices, diags = pr.evaluate(ps)
    pr.close()
    assert rc in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED)
    assert np.all(np.isfinite(prices)) and np.all(prices > 0)
