"""The binding has no CPU fallback: every public call refuses host tensors
(and int64 or non-contiguous ones) with a TypeError before anything reaches
the library. Runs without a GPU."""

import pytest
import torch

import paper_2103_15217_gb300 as etl


@pytest.fixture(autouse=True, scope="module")
def built():
    etl.build()  # the checks below run after the library loads, as they would in use


def i32(*shape):
    return torch.zeros(*shape, dtype=torch.int32)


@pytest.mark.parametrize("call", [
    lambda: etl.list_rank(i32(8), 0),
    lambda: etl.lca_preprocess(i32(8)),
    lambda: etl.lca_preprocess(i32(8), methods=("inlabel",)),
    lambda: etl.lca_preprocess_batch(i32(8), i32(3), 4),
    lambda: etl.NaiveLca(i32(8)),
    lambda: etl.find_bridges(i32(5, 2), 4),
    lambda: etl.find_bridges(i32(5, 2), 4, method="hybrid"),
    lambda: etl.find_bridges_batch(i32(5, 2), i32(2), i32(2), 4),
    lambda: etl.two_edge_cc(i32(5, 2), 4),
])
def test_host_tensors_are_refused(call):
    with pytest.raises(TypeError, match="CUDA tensor"):
        call()


def test_wrong_dtype_and_layout_are_refused():
    with pytest.raises(TypeError):
        etl._dev_i32(torch.zeros(4, dtype=torch.int64), "x")
    with pytest.raises(TypeError):
        etl._dev_i32(i32(4, 4).t(), "x")
    with pytest.raises(TypeError):
        etl._dev_i32([0, 1], "x")
    with pytest.raises(ValueError):
        etl.find_bridges(i32(6), 4)  # edges must be (m, 2)
