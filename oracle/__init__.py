"""Plain CPU oracle for RNS hybrid key switching: test infrastructure only."""
