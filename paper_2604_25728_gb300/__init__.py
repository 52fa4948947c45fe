"""SQNGD hot path on GB300 (sm_103a): C-ABI library binding."""
