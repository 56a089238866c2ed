"""The C-ABI library builds, loads without a GPU, and exports every entry
point declared in include/*.h; the binding knows all of them."""
import glob
import os
import re

import numpy as np
import pytest

from paper_2311_10337_gb300 import build as B
from paper_2311_10337_gb300 import dgec

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(dgec_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return dgec.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "dgec_run" in names and len(names) >= 8
    for n in names:
        assert hasattr(lib, n), n
    assert set(dgec.EXPORTS) >= names


def test_workspace_size_and_argument_checks(lib):
    small = dgec.workspace_size(1000, 100, 4, 5)
    big = dgec.workspace_size(100_000, 100, 4, 5)
    assert 0 < small < big
    with pytest.raises(dgec.DgecError):
        dgec.workspace_size(1000, 100, 0, 5)      # k < 1
    with pytest.raises(dgec.DgecError):
        dgec.workspace_size(1000, 100, 17, 5)     # k > 16
    with pytest.raises(dgec.DgecError):
        dgec.workspace_size(1000, 100, 4, 1)      # M < 2
    with pytest.raises(dgec.DgecError):
        dgec.workspace_size(1 << 30, 100, 4, 5)   # too many edges


def test_status_strings(lib):
    assert lib.dgec_status_string(0) == b"ok"
    assert lib.dgec_status_string(3) == b"self loop"


def test_host_arguments_are_checked_before_any_copy():
    """The host entry point copies exactly E elements from each array, so a
    wrong dtype, a strided view or a short array is rejected in the binding."""
    ok = np.zeros(5, np.int32)
    dgec._host("src", ok, np.int32, 5)
    for bad in (np.zeros(5, np.int64), np.zeros(10, np.int32)[::2], np.zeros((5, 1), np.int32),
                np.zeros(4, np.int32), [0, 0, 0, 0, 0]):
        with pytest.raises(ValueError):
            dgec._host("src", bad, np.int32, 5)
    ro = np.zeros(5, np.int32)
    ro.flags.writeable = False
    dgec._host("labels_out", ro, np.int32, 5)
    with pytest.raises(ValueError):
        dgec._host("labels_out", ro, np.int32, 5, writeable=True)


def test_device_arguments_are_checked_before_any_launch():
    """Device arguments must be contiguous 1-D CUDA tensors of the right dtype
    and length on the context's device; host tensors and numpy arrays are
    rejected (there is no CPU path)."""
    import torch
    for bad in (torch.zeros(5, dtype=torch.int32), np.zeros(5, np.int32),
                torch.zeros(5, dtype=torch.int64), torch.zeros(10, dtype=torch.int32)[::2]):
        with pytest.raises(ValueError):
            dgec._dev("src", bad, torch.int32, 5, 0)
