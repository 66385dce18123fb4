"""Register and spill budgets of the hot kernels, read from ptxas's resource report of the
sm_103a build (no GPU needed). Each budget is what a measured speed depends on:
  * the D3Q19 throughput kernel runs one 256-thread CTA per SM at <= 255 registers and must not
    spill (its z march keeps the carried differences in registers); the warp-specialised one
    launches 512 threads at 128 registers and must not spill under its register split;
  * the batch's FP32 reference tiles run 4 CTAs of 256 threads (8 of 128) per SM only at
    <= 64 registers; 72 registers cost the 64-channel batch 15%;
  * the D2Q9 throughput kernel (FP32) must not spill;
  * the adjoint's interface kernel runs 6 blocks of 128 threads per SM at <= 80 registers, and
    its cells kernel (which also carries the next reverse step's recompute) 7 blocks at <= 72 in
    FP32; neither spills, in FP32 or FP64.
A change that breaks one of them shows here before any GPU run."""
import pytest

from paper_1411_6121_gb300 import _build


@pytest.fixture(scope="module")
def res():
    _build.build()
    r = _build.resources()
    if not r:
        pytest.skip("no ptxas reports in the build folder")
    return r


def _find(res, *parts):
    hits = {k: v for k, v in res.items() if all(p in k for p in parts)}
    assert hits, parts
    return hits


def test_d3q19_warp_specialised_kernel_does_not_spill(res):
    # fused_step3d_ws<19, S, false> (the benchmark's force-free instantiation) under its register
    # split of 96 (producers) / 160 (consumers) registers
    for k, v in _find(res, "fused_step3d_wsILi19E", "Lb0E").items():
        assert v["regs"] == 128 and v["spill_stores"] == 0, (k, v)


def test_d3q19_throughput_kernel_does_not_spill(res):
    # fused_step3d<19, S, 8, FORCE> for S = float, bfloat16, half
    for k, v in _find(res, "fused_step3dILi19E", "Li8ELb").items():
        assert v["regs"] <= 255 and v["spill_stores"] == 0, (k, v)


def test_batch_fp32_tiles_fit_four_ctas_per_sm(res):
    for k, v in _find(res, "fused_step_batchILi9Ef").items():
        assert v["regs"] <= 64 and v["spill_stores"] == 0, (k, v)


def test_d2q9_throughput_kernel_fp32_does_not_spill(res):
    for k, v in _find(res, "fused_step2dIf").items():
        assert v["spill_stores"] == 0, (k, v)


def test_d3q27_throughput_kernel_spills_bounded(res):
    # at 27 velocities the force-free kernel keeps at most 64 bytes of spills (carrying the
    # x/y differences across the z march pushed it to 156)
    for k, v in _find(res, "fused_step3dILi27E", "Li8ELb0").items():
        assert v["spill_stores"] <= 64, (k, v)


def test_adjoint_kernels_fit_their_blocks_per_sm(res):
    for k, v in _find(res, "adj_faces_allIfE").items():
        assert v["regs"] <= 80 and v["spill_stores"] == 0, (k, v)
    for k, v in _find(res, "adj_cells_allIfE").items():
        assert v["regs"] <= 72 and v["spill_stores"] == 0, (k, v)
    for k, v in _find(res, "adj_faces_allIdE").items():
        assert v["spill_stores"] == 0, (k, v)
    for k, v in _find(res, "adj_cells_allIdE").items():
        assert v["spill_stores"] == 0, (k, v)
