"""ALB (adaptive load balancer, arXiv:1911.09135) graph analytics for one GB300 (sm_103a).

Submodules:
  graphgen - seeded synthetic CSR inputs (native generator).
  alb      - Python binding of the C ABI in include/alb.h (libalb.so, CUDA).
"""
__all__ = ["graphgen", "alb"]
