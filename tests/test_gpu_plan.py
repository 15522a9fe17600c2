"""rk_plan (host only) against rk_build on the GPU: with the device's opt-in
shared memory per block, the plan equals the built table's read-back in
every field but the device and its SM count."""

import pytest

from workloads import make_config, random_small

pytestmark = pytest.mark.gpu

from gpu_util import require_gpu, torch  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


from paper_1810_01051_gb300 import rk  # noqa: E402

CASES = [
    (lambda: make_config(1, n=1 << 16).patterns, {}),
    (lambda: make_config(1, n=1 << 16).patterns, dict(stages=8)),
    (lambda: make_config(1, n=1 << 16).patterns, dict(ctas_per_sm=2)),
    (lambda: make_config(2, n=1 << 16, k=3000).patterns, {}),
    (lambda: make_config(2, n=1 << 16, k=3000).patterns, dict(sample=1)),
    (lambda: random_small(2, 10, 20, 1, 3).patterns, dict(filter=rk.RK_FILTER_NONE)),
    (lambda: [b"q" * 4096, b"abcdefgh"], dict(tile_bytes=65536, stages=3)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_plan_equals_build(case):
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    optin = getattr(props, "shared_memory_per_block_optin", None)
    if not optin:
        pytest.skip("this PyTorch does not report the opt-in shared memory per block")
    make, opts = CASES[case]
    pats = make()
    plan = rk.rk_plan(pats, smem_optin=int(optin), **opts)
    t = rk.rk_build(pats, **opts)
    try:
        built = rk.rk_table_info(t)
    finally:
        rk.rk_destroy(t)
    assert built["sm_count"] == props.multi_processor_count
    for key in ("sm_count", "device"):
        plan.pop(key)
        built.pop(key)
    assert plan == built
